// Reverse mode of RCholeskyQR2 (not in the paper).  In exact arithmetic Alg. 3
// returns the unique thin QR of X (Q orthonormal, diag(R) > 0) whatever Theta
// is, so its derivative is that of the thin QR map:
//      M = R Rbar^T - Qbar^T Q,    Xbar = (Qbar + Q copyltu(M)) R^{-T},
// copyltu(M) = tril(M) + tril(M, -1)^T.  Q is recomputed by the caller from X
// and the stored R (forward substitution); this file forms Qbar^T Q (the
// cross Gram), C = copyltu(M), and row by row y = qbar + q C followed by the
// back substitution x R^T = y.  FP64 data in FP64; FP32 data with the FP32
// kernels of the mixed path (compensated cross Gram, FP32 rows).
#include <algorithm>

#include "common.cuh"
#include "rcqr_internal.h"

namespace rcqr {

int cross_gram32_groups(int64_t m, int64_t n);
cudaError_t launch_cross_gram32(const float *A, int64_t lda, const float *B, int64_t ldb, int64_t m,
                                int64_t n, double *partial, int groups, cudaStream_t st);

namespace {

constexpr int kAdjThreads = 128;

// FP64 cross Gram partials: CTA (tile, g) forms the 32 x 32 block (bi, bj) of A^T B.
__global__ void __launch_bounds__(256)
cross_gram64_kernel(const double *__restrict__ A, int64_t lda, const double *__restrict__ B, int64_t ldb,
                    int64_t m, int n, int groups, double *__restrict__ partial) {
  __shared__ double qa[64][33];
  __shared__ double qb[64][33];
  const int nb = (n + 31) / 32;
  const int bi = blockIdx.x % nb, bj = blockIdx.x / nb, g = blockIdx.y;
  const int tid = threadIdx.x, li = tid % 32, lj0 = (tid / 32) * 4;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t nt = (m + 63) / 64;
  const int64_t tb = (nt * g) / groups, te = (nt * (g + 1)) / groups;
  for (int64_t t = tb; t < te; ++t) {
    const int64_t r0 = t * 64;
    __syncthreads();
    for (int e = tid; e < 64 * 32; e += 256) {
      const int rr = e % 64, c = e / 64;
      const int64_t row = r0 + rr;
      const int ca = bi * 32 + c, cb = bj * 32 + c;
      qa[rr][c] = (row < m && ca < n) ? A[row + (int64_t)ca * lda] : 0.0;
      qb[rr][c] = (row < m && cb < n) ? B[row + (int64_t)cb * ldb] : 0.0;
    }
    __syncthreads();
    for (int rr = 0; rr < 64; ++rr) {
      const double a = qa[rr][li];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fma(a, qb[rr][lj0 + u], acc[u]);
    }
  }
  const int i = bi * 32 + li;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int j = bj * 32 + lj0 + u;
    if (i < n && j < n) partial[((int64_t)g * n + j) * n + i] = acc[u];
  }
}

// C(i, j) = sum_g partial[g](i, j): one warp per entry, fixed order.
__global__ void cross_reduce_kernel(const double *__restrict__ partial, int groups, int n, double *__restrict__ C) {
  const int64_t idx = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (idx >= (int64_t)n * n) return;
  const double s = warp_sum_strided(partial + idx, groups, (int64_t)n * n);
  if ((threadIdx.x & 31) == 0) C[idx] = s;
}

// Ct = copyltu(R Rbar^T - C) and Rt = R in the data type T; dinv = 1 / R_jj.
template <class T>
__global__ void adjoint_small_kernel(const double *__restrict__ R, int64_t ldr, const double *__restrict__ Rbar,
                                     int64_t ldrb, const double *__restrict__ C, int n, T *Ct, T *Rt, T *dinv) {
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    const int a = max(i, j), b = min(i, j);          // entry (a, b) of the lower triangle of M
    double s = 0.0;
    for (int l = a; l < n; ++l) s = fma(R[a + (int64_t)l * ldr], Rbar[b + (int64_t)l * ldrb], s);
    Ct[e] = (T)(s - C[a + (int64_t)b * n]);
    Rt[e] = (T)(i <= j ? R[i + (int64_t)j * ldr] : 0.0);
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x) dinv[j] = (T)(1.0 / R[j + (int64_t)j * ldr]);
}

// Row r: y = qbar_r + q_r Ct; then x R^T = y by back substitution; Xbar_r = x.
template <class T>
__global__ void __launch_bounds__(kAdjThreads)
adjoint_rows_kernel(const T *__restrict__ Q, int64_t ldq, const T *__restrict__ Qb, int64_t ldqb, int64_t m, int n,
                    const T *__restrict__ Ct, const T *__restrict__ Rt, const T *__restrict__ dinv, T *Xb,
                    int64_t ldxb) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= m) return;
  T q[256], y[256];
  for (int j = 0; j < n; ++j) q[j] = Q[row + (int64_t)j * ldq];
  for (int j = 0; j < n; ++j) {
    T s = Qb[row + (int64_t)j * ldqb];
    const T *cj = Ct + (int64_t)j * n;
    for (int i = 0; i < n; ++i) s = fma(q[i], cj[i], s);
    y[j] = s;
  }
  for (int j = n - 1; j >= 0; --j) {
    T s = y[j];
    for (int c = j + 1; c < n; ++c) s = fma(-Rt[j + (int64_t)c * n], y[c], s);
    y[j] = s * dinv[j];
  }
  for (int j = 0; j < n; ++j) Xb[row + (int64_t)j * ldxb] = y[j];
}

int cross_gram64_groups(int64_t m, int64_t n) {
  const int64_t nb = (n + 31) / 32;
  int64_t g = std::max<int64_t>(1, (4LL * num_sms()) / (nb * nb));
  g = std::min<int64_t>(g, std::max<int64_t>(1, (m + 63) / 64));
  return (int)std::min<int64_t>(g, 65535);
}

}  // namespace

size_t adjoint_workspace(int64_t m, int64_t n) {
  Workspace w(nullptr, 0);
  w.take<double>((size_t)std::max(cross_gram64_groups(m, n), cross_gram32_groups(m, n)) * n * n);
  w.take<double>((size_t)n * n);
  w.take<double>((size_t)n * n);
  w.take<double>((size_t)n * n);
  w.take<double>((size_t)n);
  return w.used;
}

cudaError_t launch_qr_adjoint(const void *Q, int64_t m, int64_t n, int64_t ldq, int prec, const double *R,
                              int64_t ldr, const void *Qbar, int64_t ldqb, const double *Rbar, int64_t ldrb,
                              void *Xbar, int64_t ldxb, Workspace &ws, cudaStream_t st) {
  const bool f64 = prec == RCQR_F64;
  const int groups = f64 ? cross_gram64_groups(m, n) : cross_gram32_groups(m, n);
  double *partial = ws.take<double>((size_t)groups * n * n);
  double *C = ws.take<double>((size_t)n * n);
  double *Ct = ws.take<double>((size_t)n * n);
  double *Rt = ws.take<double>((size_t)n * n);
  double *dinv = ws.take<double>((size_t)n);
  if (!partial || !C || !Ct || !Rt || !dinv) return cudaErrorMemoryAllocation;
  cudaError_t e;
  if (f64) {
    const int nb = (int)((n + 31) / 32);
    dim3 grid((unsigned)(nb * nb), (unsigned)groups);
    cross_gram64_kernel<<<grid, 256, 0, st>>>((const double *)Qbar, ldqb, (const double *)Q, ldq, m, (int)n,
                                              groups, partial);
  } else {
    e = launch_cross_gram32((const float *)Qbar, ldqb, (const float *)Q, ldq, m, n, partial, groups, st);
    if (e != cudaSuccess) return e;
  }
  cross_reduce_kernel<<<(unsigned)((n * n * 32 + 255) / 256), 256, 0, st>>>(partial, groups, (int)n, C);
  const unsigned blocks = (unsigned)((m + kAdjThreads - 1) / kAdjThreads);
  if (f64) {
    adjoint_small_kernel<double><<<1, 256, 0, st>>>(R, ldr, Rbar, ldrb, C, (int)n, Ct, Rt, dinv);
    adjoint_rows_kernel<double><<<blocks, kAdjThreads, 0, st>>>((const double *)Q, ldq, (const double *)Qbar, ldqb,
                                                                m, (int)n, Ct, Rt, dinv, (double *)Xbar, ldxb);
  } else {
    float *Ctf = reinterpret_cast<float *>(Ct), *Rtf = reinterpret_cast<float *>(Rt);
    float *dinvf = reinterpret_cast<float *>(dinv);
    adjoint_small_kernel<float><<<1, 256, 0, st>>>(R, ldr, Rbar, ldrb, C, (int)n, Ctf, Rtf, dinvf);
    adjoint_rows_kernel<float><<<blocks, kAdjThreads, 0, st>>>((const float *)Q, ldq, (const float *)Qbar, ldqb, m,
                                                               (int)n, Ctf, Rtf, dinvf, (float *)Xbar, ldxb);
  }
  return cudaGetLastError();
}

}  // namespace rcqr
