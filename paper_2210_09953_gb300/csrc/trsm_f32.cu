// The bulk steps of the mixed path (FP32 / BF16 storage) on CUDA cores in FP32,
// the working precision u of the paper's multi-precision model (Sec. 1.3,
// Sec. 5): the dominant operations at u, the small ones (sketch, QR,
// Cholesky, R products) in FP64.
//
// * Forward substitution Q = X R^{-1} (Alg. 2 step 3 / Alg. 3 step 4 / Alg. 7
//   step 4): one thread per row, the row held in registers, R rounded to FP32
//   in shared memory; q_j = (x_j - sum_{i<j} q_i R_ij) * fl(1/R_jj).  Row-wise
//   backward stable: Q (R + dR) = X with |dR| <= (n+2) u |R| (the statement
//   of Higham Thm. 8.5 that Sec. 5.1 uses, here with u = 2^-24).
// * Gram matrix A = Q^T Q (Alg. 3 step 2): FP32 products summed over 64-row
//   chunks, chunk sums added with compensated (Kahan) FP32 summation, the
//   per-CTA results added in FP64 -- about u/sqrt(m) relative, well below the
//   u of the subsequent substitution.
#include <algorithm>

#include "common.cuh"
#include "rcqr_internal.h"

namespace rcqr {

namespace {

constexpr int kT32Threads = 128;

__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 x) { return __bfloat162float(x); }

// R (n x n, FP64) -> Rf (NB x NB column-major FP32, leading rank block, zero
// padded) and dinv[j] = fl32(1 / R_jj) (0 beyond the rank).
__global__ void trsm32_prep_kernel(const double *__restrict__ R, int n, int64_t ldr,
                                   const int64_t *__restrict__ rank, int NB, float *__restrict__ Rf,
                                   float *__restrict__ dinv) {
  const int r = rank ? (int)(*rank < (int64_t)n ? *rank : (int64_t)n) : n;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int i = e % NB, j = e / NB;
    Rf[e] = (i <= j && j < r) ? __double2float_rn(R[i + (int64_t)j * ldr]) : 0.0f;
  }
  for (int j = threadIdx.x; j < NB; j += blockDim.x)
    dinv[j] = j < r ? __double2float_rn(1.0 / R[j + (int64_t)j * ldr]) : 0.0f;
}

template <class TX, int NB>
__global__ void __launch_bounds__(kT32Threads)
trsm32_kernel(const TX *__restrict__ X, int64_t m, int n, int64_t ldx, const float *__restrict__ Rf,
              const float *__restrict__ dinv, const int32_t *__restrict__ perm,
              const int64_t *__restrict__ rank, float *Q, int64_t ldq) {
  extern __shared__ float4 smem4[];
  float *Rs = reinterpret_cast<float *>(smem4);
  float *Ds = Rs + NB * NB;
  for (int e = threadIdx.x; e < NB * NB / 4; e += blockDim.x) smem4[e] = reinterpret_cast<const float4 *>(Rf)[e];
  for (int j = threadIdx.x; j < NB; j += blockDim.x) Ds[j] = dinv[j];
  __syncthreads();
  const int r = rank ? (int)(*rank < (int64_t)n ? *rank : (int64_t)n) : n;
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= m) return;
  float q[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    float v = 0.0f;
    if (j < r) {
      const int src = perm ? perm[j] : j;
      v = to_f32(X[row + (int64_t)src * ldx]);
    }
    q[j] = v;
  }
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    const float *rc = Rs + j * NB;
    float s = q[j];
#pragma unroll
    for (int i4 = 0; i4 < j / 4; ++i4) {
      const float4 rv = *reinterpret_cast<const float4 *>(rc + 4 * i4);
      s = fmaf(-q[4 * i4 + 0], rv.x, s);
      s = fmaf(-q[4 * i4 + 1], rv.y, s);
      s = fmaf(-q[4 * i4 + 2], rv.z, s);
      s = fmaf(-q[4 * i4 + 3], rv.w, s);
    }
#pragma unroll
    for (int i = (j / 4) * 4; i < j; ++i) s = fmaf(-q[i], rc[i], s);
    q[j] = s * Ds[j];
  }
#pragma unroll
  for (int j = 0; j < NB; ++j)
    if (j < n) Q[row + (int64_t)j * ldq] = q[j];
}

// ---- Gram A = Q^T Q in FP32 with compensated chunk sums
constexpr int kG32Rows = 64;     // rows per shared-memory chunk
constexpr int kG32Stride = 65;   // column stride in shared memory (conflict-free)

// CTA (tile, g): the 64 x 64 block (bi, bj) of A, bi <= bj, from row range g.
// 256 threads = 2 row-interleaved groups of 128; thread (ti, tj) of a group owns
// A entries (bi*64 + ti + 16a, bj*64 + tj + 8b), a < 4, b < 8.
__global__ void __launch_bounds__(256)
gram32_kernel(const float *__restrict__ Q, int64_t m, int n, int64_t ldq, const int64_t *__restrict__ rank,
              int groups, double *__restrict__ partial, const float *__restrict__ Q2, int64_t ldq2) {
  // two 64-column slabs of the chunk (column-major, stride 65), reused for the final reduction
  __shared__ double smd[64 * kG32Stride];
  float *qa = reinterpret_cast<float *>(smd);
  float *qb = qa + 64 * kG32Stride;
  double *red = smd;                         // 128 x 32 doubles <= 2 x 64 x 65 floats
  const int nb = (n + 63) / 64;
  // Q2 == nullptr: the Gram Q^T Q, upper tiles only; else Q^T Q2, every tile
  int bi = 0, bj = 0;
  if (Q2) {
    bi = blockIdx.x % nb;
    bj = blockIdx.x / nb;
  } else {
    int t = blockIdx.x;
    while (t >= nb - bi) {
      t -= nb - bi;
      ++bi;
    }
    bj = bi + t;
  }
  const int g = blockIdx.y;
  const int r = rank ? (int)(*rank < (int64_t)n ? *rank : (int64_t)n) : n;
  const int tid = threadIdx.x, grp = tid >> 7, lt = tid & 127;
  const int ti = lt & 15, tj = lt >> 4;
  float inner[4][8], outer[4][8], comp[4][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) outer[a][b] = comp[a][b] = 0.0f;
  const int64_t nch = (m + kG32Rows - 1) / kG32Rows;
  const int64_t cb = (nch * g) / groups, ce = (nch * (g + 1)) / groups;
  const bool diag = bi == bj && Q2 == nullptr;
  const float *qsb = diag ? qa : qb;
  const float *Qb = Q2 ? Q2 : Q;
  const int64_t ldb = Q2 ? ldq2 : ldq;
  // chunk loads: thread owns 4 row-quads (4 consecutive rows of one column) per slab,
  // prefetched into registers one chunk ahead
  float4 pa[4], pb[4];
  auto load_chunk = [&](int64_t ch) {
    const int64_t r0 = ch * kG32Rows;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int f = tid + 256 * u;
      const int c = f >> 4, rq = f & 15;
      const int64_t row = r0 + 4 * rq;
      const int ca = bi * 64 + c, cbb = bj * 64 + c;
      float va[4] = {0.f, 0.f, 0.f, 0.f}, vb[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int k4 = 0; k4 < 4; ++k4) {
        if (row + k4 < m) {
          if (ca < r) va[k4] = Q[row + k4 + (int64_t)ca * ldq];
          if (!diag && cbb < r) vb[k4] = Qb[row + k4 + (int64_t)cbb * ldb];
        }
      }
      pa[u] = make_float4(va[0], va[1], va[2], va[3]);
      pb[u] = make_float4(vb[0], vb[1], vb[2], vb[3]);
    }
  };
  if (cb < ce) load_chunk(cb);
  for (int64_t ch = cb; ch < ce; ++ch) {
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int f = tid + 256 * u;
      const int c = f >> 4, rq = f & 15;
      float *da = qa + c * kG32Stride + 4 * rq;
      da[0] = pa[u].x;
      da[1] = pa[u].y;
      da[2] = pa[u].z;
      da[3] = pa[u].w;
      if (!diag) {
        float *db = qb + c * kG32Stride + 4 * rq;
        db[0] = pb[u].x;
        db[1] = pb[u].y;
        db[2] = pb[u].z;
        db[3] = pb[u].w;
      }
    }
    __syncthreads();
    if (ch + 1 < ce) load_chunk(ch + 1);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) inner[a][b] = 0.0f;
#pragma unroll 4
    for (int rr = grp; rr < kG32Rows; rr += 2) {
      float va[4], vb[8];
#pragma unroll
      for (int a = 0; a < 4; ++a) va[a] = qa[(ti + 16 * a) * kG32Stride + rr];
#pragma unroll
      for (int b = 0; b < 8; ++b) vb[b] = qsb[(tj + 8 * b) * kG32Stride + rr];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) inner[a][b] = fmaf(va[a], vb[b], inner[a][b]);
    }
    // Kahan: outer += inner
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const float y = inner[a][b] - comp[a][b];
        const float tt = outer[a][b] + y;
        comp[a][b] = (tt - outer[a][b]) - y;
        outer[a][b] = tt;
      }
  }
  // the two groups' sums in FP64, then this CTA's block of the partial Gram
  __syncthreads();
  if (grp == 1) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) red[lt * 32 + a * 8 + b] = (double)outer[a][b] - (double)comp[a][b];
  }
  __syncthreads();
  if (grp == 0) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int i = bi * 64 + ti + 16 * a, j = bj * 64 + tj + 8 * b;
        const double v = ((double)outer[a][b] - (double)comp[a][b]) + red[lt * 32 + a * 8 + b];
        if (i < n && j < n) partial[((int64_t)g * n + j) * n + i] = v;
      }
  }
}

template <class TX>
cudaError_t launch_trsm32_t(const TX *X, int64_t m, int64_t n, int64_t ldx, const float *Rf, const float *dinv,
                            const int32_t *perm, const int64_t *rank, float *Q, int64_t ldq, int NB,
                            cudaStream_t st) {
  const unsigned blocks = (unsigned)((m + kT32Threads - 1) / kT32Threads);
  const size_t smem = (size_t)NB * NB * 4 + (size_t)NB * 4;
#define RCQR_T32(NBV)                                                                                       \
  case NBV: {                                                                                               \
    cudaError_t e = set_smem(trsm32_kernel<TX, NBV>, (int)smem);                                           \
    if (e != cudaSuccess) return e;                                                                         \
    trsm32_kernel<TX, NBV><<<blocks, kT32Threads, smem, st>>>(X, m, (int)n, ldx, Rf, dinv, perm, rank, Q, ldq); \
    break;                                                                                                  \
  }
  switch (NB) {
    RCQR_T32(16)
    RCQR_T32(32)
    RCQR_T32(48)
    RCQR_T32(64)
    RCQR_T32(80)
    RCQR_T32(96)
    RCQR_T32(112)
    RCQR_T32(128)
    default: return cudaErrorInvalidValue;
  }
#undef RCQR_T32
  return cudaGetLastError();
}

}  // namespace

bool trsm32_supported(int64_t n) { return n >= 1 && n <= 128; }

size_t trsm32_workspace(int64_t n) {
  const int NB = (int)((n + 15) / 16) * 16;
  Workspace w(nullptr, 0);
  w.take<float>((size_t)NB * NB);
  w.take<float>((size_t)NB);
  return w.used;
}

cudaError_t launch_trsm32(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, const double *R,
                          int64_t ldr, const int32_t *perm, const int64_t *rank, void *Q, int64_t ldq,
                          Workspace &ws, cudaStream_t st) {
  const int NB = (int)((n + 15) / 16) * 16;
  float *Rf = ws.take<float>((size_t)NB * NB);
  float *dinv = ws.take<float>((size_t)NB);
  if (!Rf || !dinv) return cudaErrorMemoryAllocation;
  trsm32_prep_kernel<<<1, 256, 0, st>>>(R, (int)n, ldr, rank, NB, Rf, dinv);
  if (prec == RCQR_BF16)
    return launch_trsm32_t<__nv_bfloat16>((const __nv_bfloat16 *)X, m, n, ldx, Rf, dinv, perm, rank,
                                          (float *)Q, ldq, NB, st);
  return launch_trsm32_t<float>((const float *)X, m, n, ldx, Rf, dinv, perm, rank, (float *)Q, ldq, NB, st);
}

int gram32_groups(int64_t m, int64_t n) {
  const int64_t nb = (n + 63) / 64;
  const int64_t tiles = nb * (nb + 1) / 2;
  int64_t g = std::max<int64_t>(1, (4LL * num_sms()) / tiles);
  g = std::min<int64_t>(g, std::max<int64_t>(1, (m + kG32Rows - 1) / kG32Rows));
  return (int)std::min<int64_t>(g, 65535);
}

cudaError_t launch_gram32(const float *Q, int64_t m, int64_t n, int64_t ldq, const int64_t *rank,
                          double *partial, int groups, cudaStream_t st) {
  const int64_t nb = (n + 63) / 64;
  dim3 grid((unsigned)(nb * (nb + 1) / 2), (unsigned)groups);
  gram32_kernel<<<grid, 256, 0, st>>>(Q, m, (int)n, ldq, rank, groups, partial, nullptr, 0);
  return cudaGetLastError();
}

int cross_gram32_groups(int64_t m, int64_t n) {
  const int64_t nb = (n + 63) / 64;
  int64_t g = std::max<int64_t>(1, (4LL * num_sms()) / (nb * nb));
  g = std::min<int64_t>(g, std::max<int64_t>(1, (m + kG32Rows - 1) / kG32Rows));
  return (int)std::min<int64_t>(g, 65535);
}

// partial[g] (n x n, column-major) = rows of range g of A^T B, FP32 A and B.
cudaError_t launch_cross_gram32(const float *A, int64_t lda, const float *B, int64_t ldb, int64_t m,
                                int64_t n, double *partial, int groups, cudaStream_t st) {
  const int64_t nb = (n + 63) / 64;
  dim3 grid((unsigned)(nb * nb), (unsigned)groups);
  gram32_kernel<<<grid, 256, 0, st>>>(A, m, (int)n, lda, nullptr, groups, partial, B, ldb);
  return cudaGetLastError();
}

}  // namespace rcqr
