// Forward substitution Q = X R^{-1} (Alg. 2 step 3) and the Gram matrix
// A = Q^T Q (Alg. 3 step 2) on CUDA cores in FP64 (the FP64 path), and the
// dispatch to the FP32 kernels of the mixed path (trsm_f32.cu).
//
// Substitution: the rows of X are independent (the property Sec. 5.1 uses to
// sketch the rounding errors row by row), so one thread owns one row and runs
// q_j = (x_j - sum_{i<j} q_i R_ij) / R_jj, with R staged in shared memory in
// 16-column panels.  In the rank-revealing form the input columns are
// X[:, perm[j]] for j < rank (Alg. 7 step 4) and the rest of Q is zeroed.
//
// Gram: split-K over m; CTA (b, g) forms a 32 x 32 block of A from rows of
// its range in FP64, partials are added in a fixed order.
#include <algorithm>

#include "common.cuh"
#include "rcqr_internal.h"

namespace rcqr {

namespace {

constexpr int kPanel = 16;
constexpr int kTrsmThreads = 128;

template <class TX, class TQ>
__global__ void __launch_bounds__(kTrsmThreads)
trsm_rows_kernel(const TX *__restrict__ X, int64_t m, int n, int64_t ldx, const double *__restrict__ R,
                 int64_t ldr, const int32_t *__restrict__ perm, const int64_t *__restrict__ rank,
                 TQ *Q, int64_t ldq) {
  __shared__ double Rs[256 * kPanel];
  const int r = rank ? (int)(*rank < (int64_t)n ? *rank : (int64_t)n) : n;
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double q[256];
  for (int j0 = 0; j0 < n; j0 += kPanel) {
    const int j1 = min(n, j0 + kPanel);
    __syncthreads();
    // stage R[0:j1, j0:j1] (column c at Rs[(c - j0) * 256 + i])
    for (int e = threadIdx.x; e < j1 * (j1 - j0); e += blockDim.x) {
      const int i = e % j1, c = j0 + e / j1;
      Rs[(c - j0) * 256 + i] = R[i + (int64_t)c * ldr];
    }
    __syncthreads();
    if (row < m) {
      for (int j = j0; j < j1; ++j) {
        double v = 0.0;
        if (j < r) {
          const int src = perm ? perm[j] : j;
          double s = to_f64(X[row + (int64_t)src * ldx]);
          const double *rc = Rs + (j - j0) * 256;
          for (int i = 0; i < j; ++i) s = fma(-q[i], rc[i], s);
          v = s / rc[j];
        }
        q[j] = v;
      }
    }
  }
  if (row < m) {
    for (int j = 0; j < n; ++j) Q[row + (int64_t)j * ldq] = from_f64<TQ>(q[j]);
  }
}

constexpr int kGB = 32;        // Gram block edge
constexpr int kGRows = 64;     // rows per tile

template <class TQ>
__global__ void __launch_bounds__(256)
gram_partial_kernel(const TQ *__restrict__ Q, int64_t m, int n, int64_t ldq,
                    const int64_t *__restrict__ rank, int groups, double *__restrict__ partial) {
  __shared__ double qa[kGRows][kGB + 1];
  __shared__ double qb[kGRows][kGB + 1];
  const int nb = (n + kGB - 1) / kGB;
  const int bi = blockIdx.x % nb, bj = blockIdx.x / nb;
  const int g = blockIdx.y;
  const int r = rank ? (int)(*rank < (int64_t)n ? *rank : (int64_t)n) : n;
  const int tid = threadIdx.x;
  const int li = tid % kGB, lj0 = (tid / kGB) * 4;   // 4 outputs per thread: (li, lj0..lj0+3)
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t ntiles = (m + kGRows - 1) / kGRows;
  const int64_t tb = (ntiles * g) / groups, te = (ntiles * (g + 1)) / groups;
  if (bi <= bj) {
    for (int64_t t = tb; t < te; ++t) {
      const int64_t r0 = t * kGRows;
      __syncthreads();
      for (int e = tid; e < kGRows * kGB; e += 256) {
        const int rr = e % kGRows, c = e / kGRows;
        const int64_t row = r0 + rr;
        const int ca = bi * kGB + c, cb = bj * kGB + c;
        qa[rr][c] = (row < m && ca < r) ? to_f64(Q[row + (int64_t)ca * ldq]) : 0.0;
        qb[rr][c] = (row < m && cb < r) ? to_f64(Q[row + (int64_t)cb * ldq]) : 0.0;
      }
      __syncthreads();
#pragma unroll 4
      for (int rr = 0; rr < kGRows; ++rr) {
        const double a = qa[rr][li];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = fma(a, qb[rr][lj0 + u], acc[u]);
      }
    }
  }
  const int i = bi * kGB + li;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int j = bj * kGB + lj0 + u;
    if (i < n && j < n) partial[((int64_t)g * n + j) * n + i] = acc[u];
  }
}

// A(i, j) = sum_g partial[g](min, max) (symmetric fill): one warp per entry, fixed order.
__global__ void gram_reduce_kernel(const double *__restrict__ partial, int groups, int n,
                                   double *__restrict__ A, int64_t lda) {
  const int64_t idx = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (idx >= (int64_t)n * n) return;
  int i = (int)(idx % n), j = (int)(idx / n);
  const int a = min(i, j), b = max(i, j);
  const double s = warp_sum_strided(partial + (int64_t)b * n + a, groups, (int64_t)n * n);
  if ((threadIdx.x & 31) == 0) A[i + (int64_t)j * lda] = s;
}

int gram_groups(int64_t m, int64_t n) {
  const int64_t nb = (n + kGB - 1) / kGB;
  const int64_t blocks = nb * nb;
  const int64_t target = 4LL * num_sms();
  int64_t g = std::max<int64_t>(1, target / blocks);
  g = std::min<int64_t>(g, std::max<int64_t>(1, (m + kGRows - 1) / kGRows));
  return (int)std::min<int64_t>(g, 65535);
}

}  // namespace

size_t trsm_workspace(int64_t m, int64_t n, int prec) {
  (void)m;
  if (prec == RCQR_F64) return 0;
  const size_t t = trsm32_supported(n) ? trsm32_workspace(n) : 0;
  return gemm_tc_supported(n) ? std::max(t, gemm_tc_workspace(n)) : t;
}

// FP64 X: row-wise substitution in FP64 (here).  FP32 / BF16 X: the FP32
// substitution of trsm_f32.cu, the working precision of the mixed path.
cudaError_t launch_trsm(const void *X, int64_t m, int64_t n, int64_t ldx, int prec,
                        const double *R, int64_t ldr, const int32_t *perm, const int64_t *rank,
                        void *Q, int64_t ldq, Workspace &ws, cudaStream_t st, int *dev_status) {
  (void)dev_status;
  if (prec != RCQR_F64 && trsm32_supported(n))
    return launch_trsm32(X, m, n, ldx, prec, R, ldr, perm, rank, Q, ldq, ws, st);
  if (prec != RCQR_F64) return cudaErrorInvalidValue;   // n <= 256 always takes the FP32 kernels
  const unsigned blocks = (unsigned)((m + kTrsmThreads - 1) / kTrsmThreads);
  trsm_rows_kernel<double, double><<<blocks, kTrsmThreads, 0, st>>>((const double *)X, m, (int)n, ldx, R, ldr,
                                                                     perm, rank, (double *)Q, ldq);
  return cudaGetLastError();
}

cudaError_t launch_gram_reduce(const double *partial, int groups, int64_t n, double *A, int64_t lda,
                               cudaStream_t st) {
  gram_reduce_kernel<<<(unsigned)((n * n * 32 + 255) / 256), 256, 0, st>>>(partial, groups, (int)n, A, lda);
  return cudaGetLastError();
}

// Alg. 3 steps 3-4 on a computed Q with Gram A: R' = chol(A), R <- R' R,
// Q <- Q R'^{-1} by substitution (in place).
cudaError_t launch_cholqr_pass(const double *A, int64_t n, const int64_t *rank, double *Rp, double *R, int64_t ldr,
                               void *Q, int64_t m, int64_t ldq, int qprec, Workspace &ws, cudaStream_t st,
                               int *dev_status) {
  cudaError_t e = launch_chol_update(A, n, n, rank, Rp, n, R, ldr, dev_status, st);
  if (e != cudaSuccess) return e;
  // FP32 Q: Q R'^{-1} as a tensor-core product with the explicit inverse (R' is well
  // conditioned; gemm_tc.cu); FP64 Q: the FP64 substitution
  if (qprec == RCQR_F32 && gemm_tc_supported(n))
    return launch_inverse_times((float *)Q, m, n, ldq, Rp, n, rank, dev_status, ws, st);
  return launch_trsm(Q, m, n, ldq, qprec, Rp, n, nullptr, rank, Q, ldq, ws, st, dev_status);
}

size_t gram_workspace(int64_t m, int64_t n) {
  Workspace w(nullptr, 0);
  w.take<double>((size_t)std::max(gram_groups(m, n), gram32_groups(m, n)) * n * n);
  if (gram_tc_supported(n)) return std::max(w.used, gram_tc_workspace(m, n));
  return w.used;
}

cudaError_t launch_gram(const void *Q, int64_t m, int64_t n, int64_t ldq, int prec,
                        const int64_t *rank, double *A, int64_t lda, Workspace &ws,
                        cudaStream_t st) {
  if (prec != RCQR_F64 && gram_tc_supported(n))
    return launch_gram_tc((const float *)Q, m, n, ldq, A, lda, nullptr, ws, st);   // NaN A on a timeout
  if (prec != RCQR_F64) {
    const int g32 = gram32_groups(m, n);
    double *p32 = ws.take<double>((size_t)g32 * n * n);
    if (!p32) return cudaErrorMemoryAllocation;
    cudaError_t e = launch_gram32((const float *)Q, m, n, ldq, rank, p32, g32, st);
    if (e != cudaSuccess) return e;
    gram_reduce_kernel<<<(unsigned)((n * n * 32 + 255) / 256), 256, 0, st>>>(p32, g32, (int)n, A, lda);
    return cudaGetLastError();
  }
  const int groups = gram_groups(m, n);
  double *partial = ws.take<double>((size_t)groups * n * n);
  if (!partial) return cudaErrorMemoryAllocation;
  const int nb = (int)((n + kGB - 1) / kGB);
  dim3 grid((unsigned)(nb * nb), (unsigned)groups);
  if (prec == RCQR_F64)
    gram_partial_kernel<double><<<grid, 256, 0, st>>>((const double *)Q, m, (int)n, ldq, rank,
                                                      groups, partial);
  else
    gram_partial_kernel<float><<<grid, 256, 0, st>>>((const float *)Q, m, (int)n, ldq, rank,
                                                     groups, partial);
  gram_reduce_kernel<<<(unsigned)((n * n * 32 + 255) / 256), 256, 0, st>>>(partial, groups, (int)n, A,
                                                                      lda);
  return cudaGetLastError();
}

}  // namespace rcqr
