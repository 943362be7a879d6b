// Reverse mode of RCholeskyQR2 (not in the paper).  In exact arithmetic Alg. 3
// returns the unique thin QR of X (Q orthonormal, diag(R) > 0) whatever Theta
// is, so its derivative is that of the thin QR map:
//      M = R Rbar^T - Qbar^T Q,    Xbar = (Qbar + Q copyltu(M)) R^{-T},
// copyltu(M) = tril(M) + tril(M, -1)^T.  Q is recomputed by the caller from X
// and the stored R (forward substitution); this file forms Qbar^T Q (the
// cross Gram), C = copyltu(M), Y = Qbar + Q C (a tiled product, no dependency
// along the columns), and solves Xbar R^T = Y with the library's substitution:
// reversing the order of the columns turns R^T into the upper triangular
// U = J R^T J (J the reversal), so Xbar J = (Y J) U^{-1} is the forward
// substitution of Y's reversed columns, written to Xbar's columns in reverse.
// FP64 data in FP64; FP32 data with the FP32 kernels of the mixed path.
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

// Ct = copyltu(R Rbar^T - C) in the data type T; U = J R^T J in FP64 (U(i, j) =
// R(n-1-j, n-1-i), upper triangular); rev = the reversal permutation.
template <class T>
__global__ void adjoint_small_kernel(const double *__restrict__ R, int64_t ldr, const double *__restrict__ Rbar,
                                     int64_t ldrb, const double *__restrict__ C, int n, T *Ct, double *U,
                                     int32_t *rev) {
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    const int a = max(i, j), b = min(i, j);          // entry (a, b) of the lower triangle of M
    double s = 0.0;
    for (int l = a; l < n; ++l) s = fma(R[a + (int64_t)l * ldr], Rbar[b + (int64_t)l * ldrb], s);
    Ct[e] = (T)(s - C[a + (int64_t)b * n]);
    U[e] = i <= j ? R[(n - 1 - j) + (int64_t)(n - 1 - i) * ldr] : 0.0;
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x) rev[j] = n - 1 - j;
}

// Y = Qbar + Q Ct (m x n, n <= 256): CTA tiles of 128 rows x 64 columns of Y, K in
// chunks of 32 staged in shared memory; thread (ty, tx) owns rows 8 ty .. 8 ty + 7 and
// columns 4 tx .. 4 tx + 3 of the tile (32 accumulators), every sum in the data type's
// FMA in a fixed order along K.
constexpr int kGmR = 128, kGmC = 64, kGmK = 32;
template <class T>
__global__ void __launch_bounds__(256) adjoint_gemm_kernel(const T *__restrict__ Q, int64_t ldq,
                                                          const T *__restrict__ Qb, int64_t ldqb, int64_t m, int n,
                                                          const T *__restrict__ Ct, T *__restrict__ Y, int64_t ldy) {
  __shared__ __align__(16) T As[kGmK][kGmR];
  __shared__ __align__(16) T Bs[kGmK][kGmC];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t r0 = (int64_t)blockIdx.x * kGmR;
  const int j0 = blockIdx.y * kGmC;
  T acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int k0 = 0; k0 < n; k0 += kGmK) {
    __syncthreads();
    for (int e = tid; e < kGmK * kGmR; e += 256) {
      const int rr = e % kGmR, kk = e / kGmR;
      const int64_t row = r0 + rr;
      As[kk][rr] = (row < m && k0 + kk < n) ? Q[row + (int64_t)(k0 + kk) * ldq] : T(0);
    }
    for (int e = tid; e < kGmK * kGmC; e += 256) {
      const int kk = e % kGmK, jj = e / kGmK;
      Bs[kk][jj] = (k0 + kk < n && j0 + jj < n) ? Ct[(k0 + kk) + (int64_t)(j0 + jj) * n] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kGmK; ++kk) {
      T av[8], bv[4];
#pragma unroll
      for (int a = 0; a < 8; ++a) av[a] = As[kk][8 * ty + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][4 * tx + b];
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int j = j0 + 4 * tx + b;
    if (j >= n) continue;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int64_t row = r0 + 8 * ty + a;
      if (row < m) Y[row + (int64_t)j * ldy] = Qb[row + (int64_t)j * ldqb] + acc[a][b];
    }
  }
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
  w.take<double>((size_t)n * n);                   // C
  w.take<double>((size_t)n * n);                   // Ct
  w.take<double>((size_t)n * n);                   // U
  w.take<int32_t>((size_t)n);                      // reversal
  w.take<double>((size_t)m * n);                   // Y (in the data type)
  w.take<unsigned char>(std::max(trsm_workspace(m, n, RCQR_F64), trsm_workspace(m, n, RCQR_F32)));
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
  double *U = ws.take<double>((size_t)n * n);
  int32_t *rev = ws.take<int32_t>((size_t)n);
  double *Yd = ws.take<double>((size_t)m * n);
  if (!partial || !C || !Ct || !U || !rev || !Yd) return cudaErrorMemoryAllocation;
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
  dim3 ggrid((unsigned)((m + kGmR - 1) / kGmR), (unsigned)((n + kGmC - 1) / kGmC));
  if (f64) {
    adjoint_small_kernel<double><<<1, 256, 0, st>>>(R, ldr, Rbar, ldrb, C, (int)n, Ct, U, rev);
    adjoint_gemm_kernel<double><<<ggrid, 256, 0, st>>>((const double *)Q, ldq, (const double *)Qbar, ldqb, m,
                                                       (int)n, Ct, Yd, m);
  } else {
    float *Ctf = reinterpret_cast<float *>(Ct), *Yf = reinterpret_cast<float *>(Yd);
    adjoint_small_kernel<float><<<1, 256, 0, st>>>(R, ldr, Rbar, ldrb, C, (int)n, Ctf, U, rev);
    adjoint_gemm_kernel<float><<<ggrid, 256, 0, st>>>((const float *)Q, ldq, (const float *)Qbar, ldqb, m, (int)n,
                                                      Ctf, Yf, m);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // Xbar J = (Y J) U^{-1}: the substitution reads Y's columns in reverse (perm) and writes
  // its column j to Xbar's column n-1-j (a negative leading dimension from the last column)
  char *xb = static_cast<char *>(Xbar) + (size_t)(n - 1) * ldxb * (f64 ? 8 : 4);
  return launch_trsm(Yd, m, n, m, f64 ? RCQR_F64 : RCQR_F32, U, n, rev, nullptr, xb, -ldxb, ws, st, nullptr);
}

}  // namespace rcqr
