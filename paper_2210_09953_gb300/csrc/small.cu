// Small dense FP64 kernels of the method (one CTA each; the matrices are at
// most 2048 x 256):
//  * Householder QR of the sketch P (Alg. 2 step 2; the paper's choice of
//    reflections, Sec. 3.1), diag(R) >= 0, S formed explicitly;
//  * column-pivoted Householder QR of P D^{-1}, the truncation rank and the
//    de-normalisation R <- R Pi^T D Pi (Alg. 7 steps 2, 3, 5 and Sec. 4);
//  * Cholesky of the Gram matrix with R <- R' R (Alg. 3 step 3);
//  * the inverse of an upper triangular matrix.
// The working copy of P lives in shared memory when it fits, else in the
// caller's workspace (L2 resident: at most 4 MB).
#include <algorithm>

#include "common.cuh"
#include "rcqr_internal.h"

namespace rcqr {

namespace {

constexpr int kSmallThreads = 512;
constexpr size_t kSmemLimit = 200 * 1024;

// One Householder step on column j of the k x n matrix A (column-major, lda):
// builds v in A[j:, j] (A[j,j] <- v0), returns via shared d/beta, and applies
// the reflector to columns j+1 .. n-1.
__device__ void householder_step(double *A, int k, int n, int64_t lda, int j, double *red,
                                 double *s_beta, double *s_diag) {
  double *col = A + (int64_t)j * lda;
  double tail = 0.0;
  for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) tail = fma(col[i], col[i], tail);
  tail = block_sum(tail, red);
  const double x0 = col[j];
  const double sigma = fma(x0, x0, tail);
  double beta = 0.0, d = 0.0;
  if (sigma > 0.0) {
    const double alpha = sqrt(sigma);
    const double s = x0 >= 0.0 ? 1.0 : -1.0;
    const double v0 = x0 + s * alpha;
    beta = 2.0 / fma(v0, v0, tail);
    d = -s * alpha;
    __syncthreads();
    if (threadIdx.x == 0) col[j] = v0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s_beta[j] = beta;
    s_diag[j] = d;
  }
  if (beta != 0.0) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int c = j + 1 + warp; c < n; c += nw) {
      double *ac = A + (int64_t)c * lda;
      double w = 0.0;
      for (int i = j + lane; i < k; i += 32) w = fma(col[i], ac[i], w);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      const double bw = beta * w;
      for (int i = j + lane; i < k; i += 32) ac[i] = fma(-bw, col[i], ac[i]);
    }
  }
  __syncthreads();
}

// S = H_0 ... H_{n-1} [I; 0] from the reflectors stored in A (v in A[j:, j]).
__device__ void form_S(const double *A, int k, int n, int64_t lda, const double *s_beta,
                       double *S, int64_t lds) {
  for (int e = threadIdx.x; e < k * n; e += blockDim.x) {
    const int i = e % k, c = e / k;
    S[i + (int64_t)c * lds] = (i == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = n - 1; j >= 0; --j) {
    const double beta = s_beta[j];
    if (beta != 0.0) {
      const double *v = A + (int64_t)j * lda;
      for (int c = j + warp; c < n; c += nw) {
        double *sc = S + (int64_t)c * lds;
        double w = 0.0;
        for (int i = j + lane; i < k; i += 32) w = fma(v[i], sc[i], w);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        const double bw = beta * w;
        for (int i = j + lane; i < k; i += 32) sc[i] = fma(-bw, v[i], sc[i]);
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kSmallThreads)
small_qr_kernel(const double *__restrict__ P, int k, int n, int64_t ldp, double *S, int64_t lds,
                double *R, int64_t ldr, double *gwork, int use_smem) {
  extern __shared__ double smem[];
  __shared__ double red[32];
  __shared__ double s_beta[256], s_diag[256];
  double *A = use_smem ? smem : gwork;
  const int64_t lda = k;
  for (int64_t e = threadIdx.x; e < (int64_t)k * n; e += blockDim.x) {
    const int i = (int)(e % k), c = (int)(e / k);
    A[e] = P[i + (int64_t)c * ldp];
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) householder_step(A, k, n, lda, j, red, s_beta, s_diag);
  // R with positive diagonal: row j negated when d_j < 0 (S's column j with it)
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, c = e / n;
    const double sg = s_diag[i] < 0.0 ? -1.0 : 1.0;
    double v = 0.0;
    if (i < c) v = sg * A[i + (int64_t)c * lda];
    else if (i == c) v = sg * s_diag[i];
    R[i + (int64_t)c * ldr] = v;
  }
  if (S) {
    form_S(A, k, n, lda, s_beta, S, lds);
    for (int e = threadIdx.x; e < k * n; e += blockDim.x) {
      const int i = e % k, c = e / k;
      if (s_diag[c] < 0.0) S[i + (int64_t)c * lds] = -S[i + (int64_t)c * lds];
    }
  }
}

// Column-pivoted QR of P D^{-1} + rank + de-normalised R.
__global__ void __launch_bounds__(kSmallThreads)
qrcp_kernel(const double *__restrict__ P, int k, int n, int64_t ldp, const double *colnorm2,
            double tau, double *R, int64_t ldr, int32_t *perm_out, int64_t *rank_out,
            int *dev_status, double *gwork, int use_smem) {
  extern __shared__ double smem[];
  __shared__ double red[32];
  __shared__ double s_beta[256], s_diag[256], s_norm[256], s_D[256], s_x[256], s_y[256];
  __shared__ int s_perm[256];
  __shared__ int s_piv;
  double *A = use_smem ? smem : gwork;
  const int64_t lda = k;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    double d = colnorm2 ? sqrt(colnorm2[c]) : 1.0;
    s_D[c] = d > 0.0 ? d : 1.0;
    s_perm[c] = c;
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < (int64_t)k * n; e += blockDim.x) {
    const int i = (int)(e % k), c = (int)(e / k);
    A[e] = P[i + (int64_t)c * ldp] / s_D[c];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = 0; j < n; ++j) {
    // recomputed norms of the remaining columns (rows j..k-1)
    for (int c = j + warp; c < n; c += nw) {
      const double *ac = A + (int64_t)c * lda;
      double s = 0.0;
      for (int i = j + lane; i < k; i += 32) s = fma(ac[i], ac[i], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) s_norm[c] = sqrt(s);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int p = j;
      double best = s_norm[j];
      for (int c = j + 1; c < n; ++c)
        if (s_norm[c] > best) {
          best = s_norm[c];
          p = c;
        }
      s_piv = p;
    }
    __syncthreads();
    const int p = s_piv;
    if (p != j) {
      for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const double a = A[i + (int64_t)j * lda];
        A[i + (int64_t)j * lda] = A[i + (int64_t)p * lda];
        A[i + (int64_t)p * lda] = a;
      }
      if (threadIdx.x == 0) {
        const int t = s_perm[j];
        s_perm[j] = s_perm[p];
        s_perm[p] = t;
      }
    }
    __syncthreads();
    householder_step(A, k, n, lda, j, red, s_beta, s_diag);
  }
  // R (diag >= 0) into the output buffer, then the rank test on it.
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, c = e / n;
    const double sg = s_diag[i] < 0.0 ? -1.0 : 1.0;
    double v = 0.0;
    if (i < c) v = sg * A[i + (int64_t)c * lda];
    else if (i == c) v = sg * s_diag[i];
    R[i + (int64_t)c * ldr] = v;
  }
  __syncthreads();
  // ||R||_2 by 64 steps of power iteration on R^T R from the all-ones vector.
  for (int c = threadIdx.x; c < n; c += blockDim.x) s_x[c] = 1.0;
  __syncthreads();
  double norm2 = 0.0;
  for (int it = 0; it < 64; ++it) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {  // y = R x
      double s = 0.0;
      for (int c = i; c < n; ++c) s = fma(R[i + (int64_t)c * ldr], s_x[c], s);
      s_y[i] = s;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) {  // x' = R^T y
      double s = 0.0;
      for (int i = 0; i <= c; ++i) s = fma(R[i + (int64_t)c * ldr], s_y[i], s);
      s_norm[c] = s;
    }
    __syncthreads();
    double yy = 0.0, xx = 0.0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      yy = fma(s_y[c], s_y[c], yy);
      xx = fma(s_x[c], s_x[c], xx);
    }
    yy = block_sum(yy, red);
    xx = block_sum(xx, red);
    norm2 = xx > 0.0 ? sqrt(yy / xx) : 0.0;  // ||R x|| / ||x||
    double nn = 0.0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) nn = fma(s_norm[c], s_norm[c], nn);
    nn = block_sum(nn, red);
    const double inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) s_x[c] = s_norm[c] * inv;
    __syncthreads();
  }
  // suffix Frobenius norms: F2[r] = sum_{i>=r} sum_{c>=i} R_ic^2
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    for (int c = i; c < n; ++c) s = fma(R[i + (int64_t)c * ldr], R[i + (int64_t)c * ldr], s);
    s_y[i] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double bound = tau * norm2;
    double suffix = 0.0;
    int r = n;
    // walk r from n down: suffix = F2[r]; keep the least r with sqrt(F2[r]) <= bound
    for (int rr = n; rr >= 0; --rr) {
      if (rr < n) suffix += s_y[rr];
      if (sqrt(suffix) <= bound) r = rr;
      else break;
    }
    s_piv = r;
    *rank_out = r;
    if (r == 0 && dev_status) {
      dev_status[0] = RCQR_ERANK0;
      dev_status[1] = -1;
    }
  }
  __syncthreads();
  const int r = s_piv;
  for (int c = threadIdx.x; c < n; c += blockDim.x) perm_out[c] = s_perm[c];
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, c = e / n;
    const double v = R[i + (int64_t)c * ldr];
    R[i + (int64_t)c * ldr] = (i < r) ? v * s_D[s_perm[c]] : 0.0;
  }
}

// R' = chol(A[:r,:r]); R[:r, :] <- R' R[:r, :].
__global__ void __launch_bounds__(kSmallThreads)
chol_update_kernel(const double *__restrict__ A, int n, int64_t lda, const int64_t *rank,
                   double *Rp, int64_t ldrp, double *R, int64_t ldr, int *dev_status) {
  __shared__ int s_fail;
  const int r = rank ? (int)(*rank < (int64_t)n ? *rank : (int64_t)n) : n;
  if (threadIdx.x == 0) s_fail = -1;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) Rp[(e % n) + (int64_t)(e / n) * ldrp] = 0.0;
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    __shared__ double s_d;
    if (threadIdx.x == 0) {
      double d = A[j + (int64_t)j * lda];
      for (int i = 0; i < j; ++i) d -= Rp[i + (int64_t)j * ldrp] * Rp[i + (int64_t)j * ldrp];
      if (!(d > 0.0)) {
        s_fail = j;
        s_d = 0.0;
      } else {
        s_d = sqrt(d);
        Rp[j + (int64_t)j * ldrp] = s_d;
      }
    }
    __syncthreads();
    if (s_fail >= 0) break;
    const double djj = s_d;
    for (int c = j + 1 + threadIdx.x; c < r; c += blockDim.x) {
      double s = A[j + (int64_t)c * lda];
      for (int i = 0; i < j; ++i) s -= Rp[i + (int64_t)j * ldrp] * Rp[i + (int64_t)c * ldrp];
      Rp[j + (int64_t)c * ldrp] = s / djj;
    }
    __syncthreads();
  }
  if (s_fail >= 0) {
    if (threadIdx.x == 0 && dev_status) {
      dev_status[0] = RCQR_ENOTSPD;
      dev_status[1] = s_fail;
    }
    return;
  }
  // R[:r, :] <- R' R[:r, :] in place, top row first: new row i reads rows i..r-1
  // of the old R, which later iterations have not yet overwritten; each thread
  // owns whole columns, so no other thread reads what it writes.
  for (int i = 0; i < r; ++i) {
    for (int c = i + threadIdx.x; c < n; c += blockDim.x) {
      double s = 0.0;
      const int lend = min(c, r - 1);
      for (int l = i; l <= lend; ++l) s = fma(Rp[i + (int64_t)l * ldrp], R[l + (int64_t)c * ldr], s);
      R[i + (int64_t)c * ldr] = s;
    }
    __syncthreads();
  }
}

// W = R^{-1} on the leading r x r block (zero elsewhere): column c by back substitution.
__global__ void tri_inverse_kernel(const double *__restrict__ R, int n, int64_t ldr,
                                   const int64_t *rank, double *W, int64_t ldw) {
  const int r = rank ? (int)(*rank < (int64_t)n ? *rank : (int64_t)n) : n;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    double *w = W + (int64_t)c * ldw;
    for (int i = 0; i < n; ++i) w[i] = 0.0;
    if (c >= r) continue;
    w[c] = 1.0 / R[c + (int64_t)c * ldr];
    for (int i = c - 1; i >= 0; --i) {
      double s = 0.0;
      for (int l = i + 1; l <= c; ++l) s = fma(R[i + (int64_t)l * ldr], w[l], s);
      w[i] = -s / R[i + (int64_t)i * ldr];
    }
  }
}

__global__ void reset_status_kernel(int *st) {
  st[0] = RCQR_OK;
  st[1] = -1;
}

__global__ void set_rank_kernel(int64_t *rank, int64_t v) { *rank = v; }

bool fits_smem(int64_t k, int64_t n) { return (size_t)(k * n) * 8 <= kSmemLimit; }

}  // namespace

size_t small_qr_workspace(int64_t k, int64_t n) {
  Workspace w(nullptr, 0);
  w.take<double>((size_t)k * n);
  w.take<double>((size_t)n * n);
  return w.used;
}

cudaError_t launch_small_qr(const double *P, int64_t k, int64_t n, int64_t ldp, double *S,
                            int64_t lds, double *R, int64_t ldr, Workspace &ws, cudaStream_t st) {
  const bool sm = fits_smem(k, n);
  double *g = ws.take<double>((size_t)k * n);
  if (!g) return cudaErrorMemoryAllocation;
  const size_t bytes = sm ? (size_t)k * n * 8 : 0;
  if (sm) cudaFuncSetAttribute(small_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit);
  small_qr_kernel<<<1, kSmallThreads, bytes, st>>>(P, (int)k, (int)n, ldp, S, lds, R, ldr, g, sm);
  return cudaGetLastError();
}

cudaError_t launch_qrcp(const double *P, int64_t k, int64_t n, int64_t ldp, const double *colnorm2,
                        double tau, double *R, int64_t ldr, int32_t *perm, int64_t *rank,
                        int *dev_status, Workspace &ws, cudaStream_t st) {
  const bool sm = fits_smem(k, n);
  double *g = ws.take<double>((size_t)k * n);
  if (!g) return cudaErrorMemoryAllocation;
  const size_t bytes = sm ? (size_t)k * n * 8 : 0;
  if (sm) cudaFuncSetAttribute(qrcp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit);
  qrcp_kernel<<<1, kSmallThreads, bytes, st>>>(P, (int)k, (int)n, ldp, colnorm2, tau, R, ldr, perm,
                                               rank, dev_status, g, sm);
  return cudaGetLastError();
}

cudaError_t launch_chol_update(const double *A, int64_t n, int64_t lda, const int64_t *rank,
                                  double *Rp, int64_t ldrp, double *R, int64_t ldr,
                               int *dev_status, cudaStream_t st) {
  chol_update_kernel<<<1, kSmallThreads, 0, st>>>(A, (int)n, lda, rank, Rp, ldrp, R, ldr,
                                                  dev_status);
  return cudaGetLastError();
}

cudaError_t launch_tri_inverse(const double *R, int64_t n, int64_t ldr, const int64_t *rank,
                               double *W, int64_t ldw, cudaStream_t st) {
  tri_inverse_kernel<<<1, 256, 0, st>>>(R, (int)n, ldr, rank, W, ldw);
  return cudaGetLastError();
}

cudaError_t launch_reset_status(int *dev_status, cudaStream_t st) {
  reset_status_kernel<<<1, 1, 0, st>>>(dev_status);
  return cudaGetLastError();
}

cudaError_t launch_set_rank(int64_t *rank, int64_t value, cudaStream_t st) {
  set_rank_kernel<<<1, 1, 0, st>>>(rank, value);
  return cudaGetLastError();
}

}  // namespace rcqr
