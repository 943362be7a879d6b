// Column-oriented RCholeskyQR (Alg. 4) and its randomized Gram-Schmidt form (the
// remark after Alg. 4), one block of columns per call.
//
// Block i (columns i0 .. i0+b-1, X_i given) with Q, S, R of the earlier blocks in place:
//   2.  P_i = Theta X_i                                  (the tensor-core sketch)
//   3.  R_{<i,i} = S_{<i}^+ P_i
//   4.  [S_i, R_ii] = QR(P_i - S_{<i} R_{<i,i})
// Steps 3-4 come from one Householder QR of the stacked k x (i0 + b) matrix
// [S_{<i} | P_i] = S^ R^: R_{<i,i} = R^_SS^{-1} R^_SP (back substitution) and
// (S_i, R_ii) = (S^[:, i0:], R^[i0:, i0:]); in exact arithmetic this is the least-squares
// solution and the QR of its residual (diag(R) >= 0 on both sides).
//   5.  Q_i = (X_i - Q_{<i} R_{<i,i}) R_ii^{-1}           (one thread per row, FP32 for
//       FP32/BF16 X, FP64 for FP64 X, R rounded to the working precision once)
// RGS (rgs != 0): S_i <- Theta Q_i afterwards, the sketch of the computed block.
#include <algorithm>

#include "common.cuh"
#include "rcqr_internal.h"

namespace rcqr {

namespace {

constexpr int kColThreads = 128;
constexpr int kColMaxB = 64;

// W = [S[:, :i0] | P] (k x (i0 + b), ld k).
__global__ void stack_kernel(const double *__restrict__ S, int64_t lds, int i0, const double *__restrict__ P,
                             int k, int b, double *__restrict__ W) {
  const int64_t total = (int64_t)k * (i0 + b);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % k), c = (int)(e / k);
    W[e] = c < i0 ? S[r + (int64_t)c * lds] : P[r + (int64_t)(c - i0) * k];
  }
}

// From the stacked factors: R[:i0, i0:i0+b] = Rh_SS^{-1} Rh_SP (one thread per column),
// R[i0:, i0:] = Rh_PP, rows i0.. of R[:, :i0] = 0, S[:, i0:i0+b] = Sh[:, i0:].
__global__ void scatter_kernel(const double *__restrict__ Sh, const double *__restrict__ Rh, int k, int i0, int b,
                               double *__restrict__ S, int64_t lds, double *__restrict__ R, int64_t ldr) {
  const int N = i0 + b;
  for (int c = threadIdx.x; c < b; c += blockDim.x) {
    double *out = R + (int64_t)(i0 + c) * ldr;
    for (int i = i0 - 1; i >= 0; --i) {
      double x = Rh[i + (int64_t)(i0 + c) * N];
      for (int t = i + 1; t < i0; ++t) x = fma(-Rh[i + (int64_t)t * N], out[t], x);
      out[i] = x / Rh[i + (int64_t)i * N];
    }
  }
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e % b, c = e / b;
    R[(i0 + i) + (int64_t)(i0 + c) * ldr] = i <= c ? Rh[(i0 + i) + (int64_t)(i0 + c) * N] : 0.0;
  }
  for (int e = threadIdx.x; e < b * i0; e += blockDim.x) {
    const int i = e % b, c = e / b;
    R[(i0 + i) + (int64_t)c * ldr] = 0.0;
  }
  for (int e = threadIdx.x; e < k * b; e += blockDim.x) {
    const int r = e % k, c = e / k;
    S[r + (int64_t)(i0 + c) * lds] = Sh[r + (int64_t)(i0 + c) * k];
  }
}

__device__ __forceinline__ float to_acc(float x, float) { return x; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 x, float) { return __bfloat162float(x); }
__device__ __forceinline__ double to_acc(double x, double) { return x; }

// Q_i = (X_i - Q[:, :i0] R[:i0, i0:i0+b]) R_ii^{-1}, TA the working precision.
template <class TX, class TA>
__global__ void __launch_bounds__(kColThreads) colblock_kernel(const TX *__restrict__ Xi, int64_t m, int b,
                                                              int64_t ldx, const TA *Q, int64_t ldq, int i0,
                                                              const double *__restrict__ R, int64_t ldr, TA *Qi) {
  extern __shared__ __align__(16) unsigned char col_smem[];
  TA *Rb = reinterpret_cast<TA *>(col_smem);       // i0 x b: Rb[j * b + c] = R[j, i0 + c]
  TA *Rd = Rb + (size_t)i0 * b;                    // b x b: Rd[c * b + t] = R[i0 + t, i0 + c]
  TA *Di = Rd + (size_t)b * b;                     // 1 / R_cc in the working precision
  for (int e = threadIdx.x; e < i0 * b; e += blockDim.x) {
    const int j = e / b, c = e % b;
    Rb[e] = (TA)R[j + (int64_t)(i0 + c) * ldr];
  }
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int c = e / b, t = e % b;
    Rd[e] = (TA)R[(i0 + t) + (int64_t)(i0 + c) * ldr];
  }
  for (int c = threadIdx.x; c < b; c += blockDim.x) Di[c] = (TA)(1.0 / R[(i0 + c) + (int64_t)(i0 + c) * ldr]);
  __syncthreads();
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= m) return;
  TA y[kColMaxB];
#pragma unroll
  for (int c = 0; c < kColMaxB; ++c) y[c] = c < b ? to_acc(Xi[row + (int64_t)c * ldx], TA(0)) : TA(0);
  for (int j = 0; j < i0; ++j) {
    const TA qj = Q[row + (int64_t)j * ldq];
    const TA *rb = Rb + (size_t)j * b;
#pragma unroll
    for (int c = 0; c < kColMaxB; ++c)
      if (c < b) y[c] = fma(-qj, rb[c], y[c]);
  }
#pragma unroll
  for (int c = 0; c < kColMaxB; ++c) {
    if (c < b) {
      TA s = y[c];
      const TA *rd = Rd + (size_t)c * b;
#pragma unroll
      for (int t = 0; t < c; ++t) s = fma(-y[t], rd[t], s);
      y[c] = s * Di[c];
    }
  }
#pragma unroll
  for (int c = 0; c < kColMaxB; ++c)
    if (c < b) Qi[row + (int64_t)c * ldq] = y[c];
}

}  // namespace

bool colblock_sizes_ok(int64_t m, int64_t b, int64_t k, int64_t i0) {
  return m >= 1 && b >= 1 && b <= kColMaxB && i0 >= 0 && i0 + b <= 256 && k >= i0 + b && k <= 2048 && (k % 8) == 0;
}

size_t colblock_workspace(int64_t m, int64_t b, int64_t k, int64_t i0, int prec) {
  const int64_t N = i0 + b;
  Workspace w(nullptr, 0);
  w.take<double>((size_t)k * b);      // P
  w.take<double>((size_t)k * N);      // [S | P]
  w.take<double>((size_t)k * N);      // S^
  w.take<double>((size_t)N * N);      // R^
  size_t extra = std::max(small_qr_workspace(k, N), sketch_workspace(m, b, k, 0, prec));
  extra = std::max(extra, sketch_workspace(m, b, k, 0, prec == RCQR_F64 ? RCQR_F64 : RCQR_F32));
  return ((w.used + 255) & ~size_t(255)) + extra + 256;
}

cudaError_t colblock_step(const void *Xi, int64_t m, int64_t b, int64_t ldx, int prec, int64_t k, uint64_t seed,
                          int64_t i0, int rgs, void *Q, int64_t ldq, double *S, int64_t lds, double *R, int64_t ldr,
                          Workspace &ws, cudaStream_t st, int *dev_status) {
  const int64_t N = i0 + b;
  double *P = ws.take<double>((size_t)k * b);
  double *W = ws.take<double>((size_t)k * N);
  double *Sh = ws.take<double>((size_t)k * N);
  double *Rh = ws.take<double>((size_t)N * N);
  if (!P || !W || !Sh || !Rh) return cudaErrorMemoryAllocation;
  const size_t mark = ws.used;
  cudaError_t e;
  // step 2
  if ((e = launch_sketch(Xi, m, b, ldx, prec, k, seed, 0, 0, P, k, nullptr, ws, st, dev_status)) != cudaSuccess)
    return e;
  ws.used = mark;
  // steps 3-4
  stack_kernel<<<(unsigned)std::min<int64_t>(1024, (k * N + 255) / 256), 256, 0, st>>>(S, lds, (int)i0, P, (int)k,
                                                                                       (int)b, W);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_small_qr(W, k, N, k, Sh, k, Rh, N, ws, st)) != cudaSuccess) return e;
  ws.used = mark;
  scatter_kernel<<<1, 256, 0, st>>>(Sh, Rh, (int)k, (int)i0, (int)b, S, lds, R, ldr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // step 5
  const unsigned blocks = (unsigned)((m + kColThreads - 1) / kColThreads);
  if (prec == RCQR_F64) {
    const size_t smem = ((size_t)i0 * b + (size_t)b * b + b) * sizeof(double);
    if ((e = set_smem(colblock_kernel<double, double>, (int)smem)) != cudaSuccess) return e;
    colblock_kernel<double, double><<<blocks, kColThreads, smem, st>>>(
        (const double *)Xi, m, (int)b, ldx, (const double *)Q, ldq, (int)i0, R, ldr, (double *)Q + i0 * ldq);
  } else {
    const size_t smem = ((size_t)i0 * b + (size_t)b * b + b) * sizeof(float);
    if (prec == RCQR_BF16) {
      if ((e = set_smem(colblock_kernel<__nv_bfloat16, float>, (int)smem)) != cudaSuccess) return e;
      colblock_kernel<__nv_bfloat16, float><<<blocks, kColThreads, smem, st>>>(
          (const __nv_bfloat16 *)Xi, m, (int)b, ldx, (const float *)Q, ldq, (int)i0, R, ldr, (float *)Q + i0 * ldq);
    } else {
      if ((e = set_smem(colblock_kernel<float, float>, (int)smem)) != cudaSuccess) return e;
      colblock_kernel<float, float><<<blocks, kColThreads, smem, st>>>(
          (const float *)Xi, m, (int)b, ldx, (const float *)Q, ldq, (int)i0, R, ldr, (float *)Q + i0 * ldq);
    }
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the randomized Gram-Schmidt form: S_i <- Theta Q_i
  if (rgs) {
    const int qprec = prec == RCQR_F64 ? RCQR_F64 : RCQR_F32;
    const void *Qi = prec == RCQR_F64 ? (const void *)((const double *)Q + i0 * ldq)
                                      : (const void *)((const float *)Q + i0 * ldq);
    if ((e = launch_sketch(Qi, m, b, ldq, qprec, k, seed, 0, 0, S + i0 * lds, lds, nullptr, ws, st, dev_status)) !=
        cudaSuccess)
      return e;
    ws.used = mark;
  }
  return cudaSuccess;
}

}  // namespace rcqr

using namespace rcqr;

extern "C" {

size_t rcqr_colblock_workspace_size(int64_t m, int64_t b, int64_t k, int64_t i0, int prec) {
  if (!colblock_sizes_ok(m, b, k, i0) || !(prec == RCQR_F64 || prec == RCQR_F32 || prec == RCQR_BF16)) return 0;
  return colblock_workspace(m, b, k, i0, prec);
}

rcqr_status rcqr_colblock_step(const void *Xi, int64_t m, int64_t b, int64_t ldx, int prec, int64_t k, uint64_t seed,
                               int64_t i0, int rgs, void *Q, int64_t ldq, double *S, int64_t lds, double *R,
                               int64_t ldr, void *workspace, size_t ws_bytes, int *dev_status, cudaStream_t stream) {
  if (!Xi || !Q || !S || !R || !colblock_sizes_ok(m, b, k, i0) ||
      !(prec == RCQR_F64 || prec == RCQR_F32 || prec == RCQR_BF16) || ldx < m || ldq < m || lds < k || ldr < i0 + b)
    return RCQR_EINVAL;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0 ||
      ws_bytes < colblock_workspace(m, b, k, i0, prec))
    return RCQR_EWORKSPACE;
  Workspace w(workspace, ws_bytes);
  if (dev_status && launch_reset_status(dev_status, stream) != cudaSuccess) return RCQR_ECUDA;
  const cudaError_t e = colblock_step(Xi, m, b, ldx, prec, k, seed, i0, rgs, Q, ldq, S, lds, R, ldr, w, stream,
                                      dev_status);
  if (e == cudaErrorMemoryAllocation) return RCQR_EWORKSPACE;
  return e == cudaSuccess ? RCQR_OK : RCQR_ECUDA;
}

rcqr_status rcqr_factor_colwise(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, int64_t k, uint64_t seed,
                                int64_t b, int rgs, void *Q, int64_t ldq, double *S, int64_t lds, double *R,
                                int64_t ldr, void *workspace, size_t ws_bytes, int *dev_status, cudaStream_t stream) {
  if (!X || n < 1 || b < 1 || b > n || !colblock_sizes_ok(m, std::min(b, n), k, n - std::min(b, n)) || ldr < n)
    return RCQR_EINVAL;
  // the workspace of the largest step
  size_t need = 0;
  for (int64_t i0 = 0; i0 < n; i0 += b) need = std::max(need, colblock_workspace(m, std::min(b, n - i0), k, i0, prec));
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0 || ws_bytes < need) return RCQR_EWORKSPACE;
  if (dev_status && launch_reset_status(dev_status, stream) != cudaSuccess) return RCQR_ECUDA;
  const size_t es = elem_size(prec);
  for (int64_t i0 = 0; i0 < n; i0 += b) {
    const int64_t bi = std::min(b, n - i0);
    Workspace w(workspace, ws_bytes);
    const cudaError_t e = colblock_step(static_cast<const char *>(X) + (size_t)i0 * ldx * es, m, bi, ldx, prec, k,
                                        seed, i0, rgs, Q, ldq, S, lds, R, ldr, w, stream, dev_status);
    if (e == cudaErrorMemoryAllocation) return RCQR_EWORKSPACE;
    if (e != cudaSuccess) return RCQR_ECUDA;
  }
  return RCQR_OK;
}

}  // extern "C"
