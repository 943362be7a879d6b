// The implicit Q factor of RCholeskyQR2 (the remark after Alg. 3): step 4,
// Q <- Q1 R'^{-1}, is skipped; Q is kept as the pair (Q1, R') and applied through
// its products, Q Y = Q1 (R'^{-1} Y) and Q^T B = R'^{-T} (Q1^T B).  Both are
// stable because Q1 and R' are well conditioned (Sec. 3.1).
//
// * q_times: W = R'^{-1} Y (n x c, FP64 back substitution, one thread per column),
//   then Z = Q1 W with one thread per row of Q1 and W in shared memory (in Q1's
//   precision: FP64 for F64, FP32 for F32).
// * qt_times: per-CTA partial sums of Q1^T B over row ranges (16-row chunks staged in
//   shared memory, products accumulated in FP64), a fixed-order reduction, and
//   Z = R'^{-T} C by forward substitution, one thread per column.
// Limits: n, c <= 256 and n * c <= 8192 (shared memory: 16 (n + c) or n c doubles).
#include <algorithm>

#include "common.cuh"
#include "rcqr_internal.h"

namespace rcqr {

namespace {

constexpr int kImpRows = 128;          // rows per CTA in q_times
constexpr int kImpThreads = 256;       // qt_times
constexpr int kImpChunk = 16;          // rows per shared-memory chunk in qt_times
constexpr int kImpPairs = 32;          // (j, c) pairs per thread in qt_times (n c <= 8192)

__global__ void rinv_cols_kernel(const double *__restrict__ Rp, int n, int64_t ldrp, const double *__restrict__ Y,
                                 int64_t ldy, int c, double *__restrict__ W) {
  for (int cc = threadIdx.x; cc < c; cc += blockDim.x) {
    double *w = W + (int64_t)cc * n;
    for (int i = n - 1; i >= 0; --i) {
      double x = Y[i + (int64_t)cc * ldy];
      for (int t = i + 1; t < n; ++t) x = fma(-Rp[i + (int64_t)t * ldrp], w[t], x);
      w[i] = x / Rp[i + (int64_t)i * ldrp];
    }
  }
}

template <class TQ>
__global__ void __launch_bounds__(kImpRows) q_times_kernel(const TQ *__restrict__ Q, int64_t m, int n, int64_t ldq,
                                                          const double *__restrict__ W, int c, TQ *__restrict__ Z,
                                                          int64_t ldz) {
  extern __shared__ __align__(16) unsigned char imp_smem[];
  TQ *Ws = reinterpret_cast<TQ *>(imp_smem);
  for (int e = threadIdx.x; e < n * c; e += blockDim.x) Ws[e] = (TQ)W[e];
  __syncthreads();
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= m) return;
  for (int cc = 0; cc < c; ++cc) {
    TQ acc = TQ(0);
    for (int j = 0; j < n; ++j) acc = fma(Q[row + (int64_t)j * ldq], Ws[j + cc * n], acc);
    Z[row + (int64_t)cc * ldz] = acc;
  }
}

template <class TQ>
__global__ void __launch_bounds__(kImpThreads) qt_times_kernel(const TQ *__restrict__ Q, int64_t ldq,
                                                              const TQ *__restrict__ B, int64_t ldb, int64_t m, int n,
                                                              int c, int groups, double *__restrict__ partial) {
  extern __shared__ __align__(16) unsigned char imp_smem[];
  double *qs = reinterpret_cast<double *>(imp_smem);           // kImpChunk x n, row-major: qs[rr * n + j]
  double *bs = qs + kImpChunk * n;                               // kImpChunk x c: bs[rr * c + cc]
  const int g = blockIdx.x;
  const int64_t nch = (m + kImpChunk - 1) / kImpChunk;
  const int64_t cb = nch * g / groups, ce = nch * (g + 1) / groups;
  const int pairs = n * c;
  double acc[kImpPairs];
#pragma unroll
  for (int p = 0; p < kImpPairs; ++p) acc[p] = 0.0;
  for (int64_t ch = cb; ch < ce; ++ch) {
    const int64_t r0 = ch * kImpChunk;
    for (int e = threadIdx.x; e < kImpChunk * n; e += blockDim.x) {
      const int rr = e % kImpChunk, j = e / kImpChunk;
      qs[rr * n + j] = r0 + rr < m ? (double)Q[r0 + rr + (int64_t)j * ldq] : 0.0;
    }
    for (int e = threadIdx.x; e < kImpChunk * c; e += blockDim.x) {
      const int rr = e % kImpChunk, cc = e / kImpChunk;
      bs[rr * c + cc] = r0 + rr < m ? (double)B[r0 + rr + (int64_t)cc * ldb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < kImpPairs; ++p) {
      const int pi = threadIdx.x + p * kImpThreads;
      if (pi < pairs) {
        const int j = pi % n, cc = pi / n;
        double s = acc[p];
#pragma unroll
        for (int rr = 0; rr < kImpChunk; ++rr) s = fma(qs[rr * n + j], bs[rr * c + cc], s);
        acc[p] = s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < kImpPairs; ++p) {
    const int pi = threadIdx.x + p * kImpThreads;
    if (pi < pairs) partial[(int64_t)g * pairs + pi] = acc[p];
  }
}

// C = sum_g partial[g] (fixed order, one thread per entry), then Z = R'^{-T} C column by column.
__global__ void qt_finish_kernel(const double *__restrict__ partial, int groups, int n, int c,
                                 const double *__restrict__ Rp, int64_t ldrp, double *__restrict__ C,
                                 double *__restrict__ Z, int64_t ldz) {
  const int pairs = n * c;
  for (int e = threadIdx.x; e < pairs; e += blockDim.x) {
    double s = 0.0;
    for (int g = 0; g < groups; ++g) s += partial[(int64_t)g * pairs + e];
    C[e] = s;
  }
  __syncthreads();
  for (int cc = threadIdx.x; cc < c; cc += blockDim.x) {
    // R'^T z = C[:, cc]: z_j = (C_j - sum_{i<j} R'_{ij} z_i) / R'_{jj}
    for (int j = 0; j < n; ++j) {
      double x = C[j + cc * n];
      for (int i = 0; i < j; ++i) x = fma(-Rp[i + (int64_t)j * ldrp], Z[i + (int64_t)cc * ldz], x);
      Z[j + (int64_t)cc * ldz] = x / Rp[j + (int64_t)j * ldrp];
    }
  }
}

int qt_groups(int64_t m) {
  const int64_t chunks = (m + kImpChunk - 1) / kImpChunk;
  return (int)std::max<int64_t>(1, std::min<int64_t>(chunks, 2LL * num_sms()));
}

}  // namespace

bool implicit_sizes_ok(int64_t n, int64_t c) { return n >= 1 && n <= 256 && c >= 1 && c <= 256 && n * c <= 8192; }

size_t implicit_workspace(int64_t m, int64_t n, int64_t c) {
  Workspace w(nullptr, 0);
  w.take<double>((size_t)n * c);                       // W or C
  w.take<double>((size_t)qt_groups(m) * n * c);        // partial sums
  return w.used;
}

cudaError_t launch_implicit_q_times(const void *Q, int64_t m, int64_t n, int64_t ldq, int prec, const double *Rp,
                                    int64_t ldrp, const double *Y, int64_t ldy, int64_t c, void *Z, int64_t ldz,
                                    Workspace &ws, cudaStream_t st) {
  double *W = ws.take<double>((size_t)n * c);
  if (!W) return cudaErrorMemoryAllocation;
  rinv_cols_kernel<<<1, 256, 0, st>>>(Rp, (int)n, ldrp, Y, ldy, (int)c, W);
  const unsigned blocks = (unsigned)((m + kImpRows - 1) / kImpRows);
  if (prec == RCQR_F64) {
    const size_t smem = (size_t)n * c * sizeof(double);
    cudaError_t e = set_smem(q_times_kernel<double>, (int)smem);
    if (e != cudaSuccess) return e;
    q_times_kernel<double><<<blocks, kImpRows, smem, st>>>((const double *)Q, m, (int)n, ldq, W, (int)c, (double *)Z,
                                                            ldz);
  } else {
    const size_t smem = (size_t)n * c * sizeof(float);
    cudaError_t e = set_smem(q_times_kernel<float>, (int)smem);
    if (e != cudaSuccess) return e;
    q_times_kernel<float><<<blocks, kImpRows, smem, st>>>((const float *)Q, m, (int)n, ldq, W, (int)c, (float *)Z,
                                                           ldz);
  }
  return cudaGetLastError();
}

cudaError_t launch_implicit_qt_times(const void *Q, int64_t m, int64_t n, int64_t ldq, int prec, const double *Rp,
                                     int64_t ldrp, const void *B, int64_t ldb, int64_t c, double *Z, int64_t ldz,
                                     Workspace &ws, cudaStream_t st) {
  double *C = ws.take<double>((size_t)n * c);
  const int G = qt_groups(m);
  double *partial = ws.take<double>((size_t)G * n * c);
  if (!C || !partial) return cudaErrorMemoryAllocation;
  const size_t smem = (size_t)kImpChunk * (n + c) * sizeof(double);
  cudaError_t e;
  if (prec == RCQR_F64) {
    if ((e = set_smem(qt_times_kernel<double>, (int)smem)) != cudaSuccess) return e;
    qt_times_kernel<double><<<G, kImpThreads, smem, st>>>((const double *)Q, ldq, (const double *)B, ldb, m, (int)n,
                                                           (int)c, G, partial);
  } else {
    if ((e = set_smem(qt_times_kernel<float>, (int)smem)) != cudaSuccess) return e;
    qt_times_kernel<float><<<G, kImpThreads, smem, st>>>((const float *)Q, ldq, (const float *)B, ldb, m, (int)n,
                                                          (int)c, G, partial);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  qt_finish_kernel<<<1, 256, 0, st>>>(partial, G, (int)n, (int)c, Rp, ldrp, C, Z, ldz);
  return cudaGetLastError();
}

}  // namespace rcqr
