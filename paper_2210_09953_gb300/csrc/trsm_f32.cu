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

// RR rows per thread (RR = 2 for NB <= 64): every R value read from shared
// memory (a broadcast) serves RR rows, so the shared-memory traffic per FMA is
// 1 / RR of the one-row form.  Rows row0 + t * kT32Threads, t < RR.
template <class TX, int NB, int RR>
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
  const int64_t row0 = (int64_t)blockIdx.x * (RR * kT32Threads) + threadIdx.x;
  if (row0 >= m) return;
  bool live[RR];
#pragma unroll
  for (int t = 0; t < RR; ++t) live[t] = row0 + (int64_t)t * kT32Threads < m;
  float q[RR][NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    const int src = (perm && j < r) ? perm[j] : j;
#pragma unroll
    for (int t = 0; t < RR; ++t)
      q[t][j] = (j < r && live[t]) ? to_f32(X[row0 + (int64_t)t * kT32Threads + (int64_t)src * ldx]) : 0.0f;
  }
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    const float *rc = Rs + j * NB;
    float s[RR];
#pragma unroll
    for (int t = 0; t < RR; ++t) s[t] = q[t][j];
#pragma unroll
    for (int i4 = 0; i4 < j / 4; ++i4) {
      const float4 rv = *reinterpret_cast<const float4 *>(rc + 4 * i4);
#pragma unroll
      for (int t = 0; t < RR; ++t) {
        s[t] = fmaf(-q[t][4 * i4 + 0], rv.x, s[t]);
        s[t] = fmaf(-q[t][4 * i4 + 1], rv.y, s[t]);
        s[t] = fmaf(-q[t][4 * i4 + 2], rv.z, s[t]);
        s[t] = fmaf(-q[t][4 * i4 + 3], rv.w, s[t]);
      }
    }
#pragma unroll
    for (int i = (j / 4) * 4; i < j; ++i) {
      const float rvi = rc[i];
#pragma unroll
      for (int t = 0; t < RR; ++t) s[t] = fmaf(-q[t][i], rvi, s[t]);
    }
    const float dj = Ds[j];
#pragma unroll
    for (int t = 0; t < RR; ++t) q[t][j] = s[t] * dj;
  }
  // the store addresses are recomputed from an opaque copy of ldq rather than kept
  // live from the loads (2 NB 64-bit addresses would cost 4 NB registers)
  int64_t lds = ldq;
  asm volatile("" : "+l"(lds));
#pragma unroll
  for (int j = 0; j < NB; ++j)
    if (j < n)
#pragma unroll
      for (int t = 0; t < RR; ++t)
        if (live[t]) Q[row0 + (int64_t)t * kT32Threads + (int64_t)j * lds] = q[t][j];
}

// ---- Wide R (64 < n <= 256): the row's columns in panels of 64.  A panel is
// first updated by the earlier panels -- the row's earlier q, re-read from Q
// (just written by this thread, L2-resident), times a 64 x 64 block of R: 64
// independent FMA chains per thread -- and then solved against its diagonal
// block (the triangular part).  Same backward error bound as the row kernel.
constexpr int kWide = 64;

template <class TX>
__global__ void __launch_bounds__(kT32Threads)
trsm32_wide_kernel(const TX *__restrict__ X, int64_t m, int n, int64_t ldx, const float *__restrict__ Rf, int NB,
                   const float *__restrict__ dinv, const int32_t *__restrict__ perm,
                   const int64_t *__restrict__ rank, float *Q, int64_t ldq) {
  __shared__ __align__(16) float Rb[kWide * kWide];   // off-diagonal block, row-major: Rb[i * 64 + c]
  __shared__ __align__(16) float Rd[kWide * kWide];   // diagonal block, column-major: Rd[c * 64 + i]
  __shared__ float Ds[kWide];
  const int r = rank ? (int)(*rank < (int64_t)n ? *rank : (int64_t)n) : n;
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = row < m;
  const int NP = (n + kWide - 1) / kWide;
  for (int P = 0; P < NP; ++P) {
    const int c0 = P * kWide;
    float acc[kWide];
#pragma unroll
    for (int c = 0; c < kWide; ++c) {
      const int j = c0 + c;
      acc[c] = 0.0f;
      if (live && j < r) acc[c] = to_f32(X[row + (int64_t)(perm ? perm[j] : j) * ldx]);
    }
    for (int p = 0; p < P; ++p) {
      __syncthreads();
      for (int e = threadIdx.x; e < kWide * kWide; e += blockDim.x) {
        const int i = e / kWide, c = e % kWide;
        Rb[e] = Rf[(p * kWide + i) + (int64_t)(c0 + c) * NB];
      }
      __syncthreads();
#pragma unroll 4
      for (int i = 0; i < kWide; ++i) {
        const float qi = live ? Q[row + (int64_t)(p * kWide + i) * ldq] : 0.0f;
        const float4 *rb = reinterpret_cast<const float4 *>(Rb + i * kWide);
#pragma unroll
        for (int c4 = 0; c4 < kWide / 4; ++c4) {
          const float4 rv = rb[c4];
          acc[4 * c4 + 0] = fmaf(-qi, rv.x, acc[4 * c4 + 0]);
          acc[4 * c4 + 1] = fmaf(-qi, rv.y, acc[4 * c4 + 1]);
          acc[4 * c4 + 2] = fmaf(-qi, rv.z, acc[4 * c4 + 2]);
          acc[4 * c4 + 3] = fmaf(-qi, rv.w, acc[4 * c4 + 3]);
        }
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kWide * kWide; e += blockDim.x) {
      const int c = e / kWide, i = e % kWide;
      Rd[e] = Rf[(c0 + i) + (int64_t)(c0 + c) * NB];
    }
    for (int c = threadIdx.x; c < kWide; c += blockDim.x) Ds[c] = dinv[c0 + c];
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kWide; ++c) {
      const float *rc = Rd + c * kWide;
      float sres = acc[c];
#pragma unroll
      for (int i4 = 0; i4 < c / 4; ++i4) {
        const float4 rv = *reinterpret_cast<const float4 *>(rc + 4 * i4);
        sres = fmaf(-acc[4 * i4 + 0], rv.x, sres);
        sres = fmaf(-acc[4 * i4 + 1], rv.y, sres);
        sres = fmaf(-acc[4 * i4 + 2], rv.z, sres);
        sres = fmaf(-acc[4 * i4 + 3], rv.w, sres);
      }
#pragma unroll
      for (int i = (c / 4) * 4; i < c; ++i) sres = fmaf(-acc[i], rc[i], sres);
      acc[c] = sres * Ds[c];
    }
    if (live) {
#pragma unroll
      for (int c = 0; c < kWide; ++c)
        if (c0 + c < n) Q[row + (int64_t)(c0 + c) * ldq] = acc[c];
    }
  }
}

// ---- Substitution fused with the Gram of the second pass (Alg. 2 step 3 and
// Alg. 3 step 2, mixed path, NB <= 64).  A persistent CTA takes tiles of 256
// rows: two rows per thread are substituted as in trsm32_kernel, written to Q
// and to a shared tile, and the CTA's partial Q^T Q is accumulated from the
// tile in 32-row FP32 chunks with compensated chunk sums -- the arithmetic of
// gram32_kernel -- so Q is not read back from memory.
//
// Only the upper triangle of Q^T Q is needed.  In 8-row strips (strip s: rows
// 8s..8s+7, columns 8s..63), warp w takes strips w and 7 - w, whose widths add
// up to 72 columns.  One code path serves all warps (the instruction cache
// holds one copy): lane (p, c) owns rows 2p, 2p + 1 of both strips and columns
// c + 8u of each, u < 8 in strip w and u < 4 in strip 7 - w; columns past 63
// wrap to columns below the strip's diagonal block, computed but not stored.
// That is 96 of the 128 multiply-adds per row and lane of the full product.
// The tile is column-major with a stride of 4 words mod 32 banks, so each
// operand load of a warp (8 distinct columns, or 4 distinct rows) is one
// conflict-free wavefront.
constexpr int kTGRows = 2 * kT32Threads;      // rows per tile
constexpr int kTGStride = kTGRows + 4;        // tile column stride (16-byte aligned rows)
constexpr int kTGG1 = 8, kTGG2 = 4;           // column groups per lane in the two strips
constexpr int kTGG = kTGG1 + kTGG2;

struct TgLane {
  int arow[2][2];     // [strip][h]: tile column of the lane's rows
  int bcol[kTGG];     // tile column of group u (strip 1: u < kTGG1)
};

__device__ __forceinline__ TgLane tg_lane(int w, int p, int c) {
  TgLane L;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    L.arow[0][h] = 8 * w + 2 * p + h;
    L.arow[1][h] = 8 * (7 - w) + 2 * p + h;
  }
#pragma unroll
  for (int u = 0; u < kTGG1; ++u) L.bcol[u] = (8 * w + 8 * u + c) & 63;
#pragma unroll
  for (int u = 0; u < kTGG2; ++u) L.bcol[kTGG1 + u] = (8 * (7 - w) + 8 * u + c) & 63;
  return L;
}

template <class TX, int NB>
__global__ void __launch_bounds__(kT32Threads)
trsm32_gram_kernel(const TX *__restrict__ X, int64_t m, int n, int64_t ldx, const float *__restrict__ Rf,
                   const float *__restrict__ dinv, const int32_t *__restrict__ perm,
                   const int64_t *__restrict__ rank, float *Q, int64_t ldq, double *__restrict__ partial) {
  static_assert(NB <= 64, "one 64 x 64 Gram tile");
  extern __shared__ float4 tg_smem4[];
  float *Rs = reinterpret_cast<float *>(tg_smem4);
  float *Ds = Rs + NB * NB;
  float *Ts = Ds + 64;                         // 64 columns x kTGStride (columns >= NB stay zero)
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * NB / 4; e += blockDim.x) tg_smem4[e] = reinterpret_cast<const float4 *>(Rf)[e];
  for (int j = tid; j < 64; j += blockDim.x) Ds[j] = j < NB ? dinv[j] : 0.0f;
  for (int e = tid; e < 64 * kTGStride; e += blockDim.x) Ts[e] = 0.0f;
  __syncthreads();
  const int r = rank ? (int)(*rank < (int64_t)n ? *rank : (int64_t)n) : n;
  const TgLane L = tg_lane(tid >> 5, tid & 3, (tid >> 2) & 7);
  float outer[2][kTGG], comp[2][kTGG];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int u = 0; u < kTGG; ++u) outer[h][u] = comp[h][u] = 0.0f;
  const int64_t tiles = (m + kTGRows - 1) / kTGRows;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t row0 = tile * kTGRows + tid;
    {
      bool live[2];
      live[0] = row0 < m;
      live[1] = row0 + kT32Threads < m;
      float q[2][NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const int src = (perm && j < r) ? perm[j] : j;
#pragma unroll
        for (int t = 0; t < 2; ++t)
          q[t][j] = (j < r && live[t]) ? to_f32(X[row0 + (int64_t)t * kT32Threads + (int64_t)src * ldx]) : 0.0f;
      }
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const float *rc = Rs + j * NB;
        float s[2] = {q[0][j], q[1][j]};
#pragma unroll
        for (int i4 = 0; i4 < j / 4; ++i4) {
          const float4 rv = *reinterpret_cast<const float4 *>(rc + 4 * i4);
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            s[t] = fmaf(-q[t][4 * i4 + 0], rv.x, s[t]);
            s[t] = fmaf(-q[t][4 * i4 + 1], rv.y, s[t]);
            s[t] = fmaf(-q[t][4 * i4 + 2], rv.z, s[t]);
            s[t] = fmaf(-q[t][4 * i4 + 3], rv.w, s[t]);
          }
        }
#pragma unroll
        for (int i = (j / 4) * 4; i < j; ++i) {
          const float rvi = rc[i];
#pragma unroll
          for (int t = 0; t < 2; ++t) s[t] = fmaf(-q[t][i], rvi, s[t]);
        }
        const float dj = Ds[j];
#pragma unroll
        for (int t = 0; t < 2; ++t) q[t][j] = s[t] * dj;
      }
#pragma unroll
      for (int j = 0; j < NB; ++j) {
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          if (j < n && live[t]) Q[row0 + (int64_t)t * kT32Threads + (int64_t)j * ldq] = q[t][j];
          Ts[j * kTGStride + tid + t * kT32Threads] = q[t][j];
        }
      }
    }
    __syncthreads();
    // partial Gram of the tile (upper triangle): eight 32-row chunks, each summed in FP32
    // and added compensated
#pragma unroll 1
    for (int c0 = 0; c0 < kTGRows; c0 += 32) {
      float inner[2][kTGG];
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int u = 0; u < kTGG; ++u) inner[h][u] = 0.0f;
#pragma unroll 2
      for (int s4 = 0; s4 < 8; ++s4) {
        const int rr = c0 + 4 * s4;
        float4 a[2][2], b[kTGG];
#pragma unroll
        for (int st = 0; st < 2; ++st)
#pragma unroll
          for (int h = 0; h < 2; ++h) a[st][h] = *reinterpret_cast<const float4 *>(Ts + L.arow[st][h] * kTGStride + rr);
#pragma unroll
        for (int u = 0; u < kTGG; ++u) b[u] = *reinterpret_cast<const float4 *>(Ts + L.bcol[u] * kTGStride + rr);
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int u = 0; u < kTGG; ++u) {
            const float4 av = a[u < kTGG1 ? 0 : 1][h];
            inner[h][u] = fmaf(av.x, b[u].x, inner[h][u]);
            inner[h][u] = fmaf(av.y, b[u].y, inner[h][u]);
            inner[h][u] = fmaf(av.z, b[u].z, inner[h][u]);
            inner[h][u] = fmaf(av.w, b[u].w, inner[h][u]);
          }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int u = 0; u < kTGG; ++u) {
          const float y = inner[h][u] - comp[h][u];
          const float tt = outer[h][u] + y;
          comp[h][u] = (tt - outer[h][u]) - y;
          outer[h][u] = tt;
        }
    }
    __syncthreads();   // the tile is rewritten by the next iteration
  }
  // entries i <= j only: the reduction reads the upper triangle of every partial
  double *pb = partial + (int64_t)blockIdx.x * n * n;
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int u = 0; u < kTGG; ++u) {
      const int i = L.arow[u < kTGG1 ? 0 : 1][h], j = L.bcol[u];
      if (i <= j && j < n) pb[(int64_t)j * n + i] = (double)outer[h][u] - (double)comp[h][u];
    }
}

// ---- Gram A = Q^T Q in FP32 with compensated chunk sums
constexpr int kG32Rows = 64;     // rows per shared-memory chunk
constexpr int kG32Stride = 68;   // column stride in shared memory (16-byte rows, conflict-free quads)

constexpr int kG32Stages = 3;    // chunks in flight (cp.async ring)
constexpr int kG32Slab = 64 * kG32Stride;   // floats per 64-column slab of a chunk

__device__ __forceinline__ void cp_async16_zfill(void *dst, const void *src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}

// CTA (tile, g): the 64 x 64 block (bi, bj) of A, bi <= bj, from row range g.
// 256 threads = 2 groups of 128 that take the two 32-row halves of each
// 64-row chunk; thread (ti, tj) of a group owns A entries
// (bi*64 + ti + 16a, bj*64 + tj + 8b), a < 4, b < 8.  Chunks stream through a
// ring of kG32Stages shared-memory slots (cp.async, 16 bytes = 4 rows of one
// column per copy; `vec` = false falls back to plain loads).  Four rows of a
// column are read at once (16-byte loads).
__global__ void __launch_bounds__(256)
gram32_kernel(const float *__restrict__ Q, int64_t m, int n, int64_t ldq, const int64_t *__restrict__ rank,
              int groups, double *__restrict__ partial, const float *__restrict__ Q2, int64_t ldq2, int vec) {
  extern __shared__ float4 g32_smem4[];
  float *ring = reinterpret_cast<float *>(g32_smem4);
  double *red = reinterpret_cast<double *>(g32_smem4);   // 128 x 32 doubles, reused at the end
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
  const int slabs = diag ? 1 : 2;
  const float *Qb = Q2 ? Q2 : Q;
  const int64_t ldb = Q2 ? ldq2 : ldq;
  // copies chunk ch into ring slot `slot`: (slab, column c, row quad rq) per 16 bytes
  auto issue = [&](int64_t ch, int slot) {
    const int64_t r0 = ch * kG32Rows;
    for (int f = tid; f < slabs * 1024; f += 256) {
      const int sl = f >> 10, c = (f >> 4) & 63, rq = f & 15;
      const int col = (sl == 0 ? bi : bj) * 64 + c;
      const float *base = sl == 0 ? Q : Qb;
      const int64_t ld = sl == 0 ? ldq : ldb;
      const int64_t row = r0 + 4 * rq;
      float *dst = ring + (slot * 2 + sl) * kG32Slab + c * kG32Stride + 4 * rq;
      const int64_t left = m - row;
      const int valid = (col < r && left > 0) ? (int)(left < 4 ? left : 4) : 0;
      if (vec) {
        const float *src = valid > 0 ? base + row + (int64_t)col * ld : base;
        cp_async16_zfill(dst, src, 4 * valid);
      } else {
        float v[4];
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4) v[k4] = k4 < valid ? base[row + k4 + (int64_t)col * ld] : 0.0f;
        *reinterpret_cast<float4 *>(dst) = make_float4(v[0], v[1], v[2], v[3]);
      }
    }
  };
#pragma unroll 1
  for (int s0 = 0; s0 < kG32Stages - 1; ++s0) {
    if (cb + s0 < ce) issue(cb + s0, (int)((cb + s0) % kG32Stages));
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  for (int64_t ch = cb; ch < ce; ++ch) {
    const int64_t ahead = ch + kG32Stages - 1;
    if (ahead < ce) issue(ahead, (int)(ahead % kG32Stages));
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group %0;" ::"n"(kG32Stages - 1) : "memory");
    __syncthreads();
    const int slot = (int)(ch % kG32Stages);
    const float *qa = ring + (slot * 2) * kG32Slab;
    const float *qsb = diag ? qa : qa + kG32Slab;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) inner[a][b] = 0.0f;
#pragma unroll 2
    for (int s = 0; s < 8; ++s) {
      const int rr = 32 * grp + 4 * s;
      float4 va[4], vb[8];
#pragma unroll
      for (int a = 0; a < 4; ++a) va[a] = *reinterpret_cast<const float4 *>(qa + (ti + 16 * a) * kG32Stride + rr);
#pragma unroll
      for (int b = 0; b < 8; ++b) vb[b] = *reinterpret_cast<const float4 *>(qsb + (tj + 8 * b) * kG32Stride + rr);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          inner[a][b] = fmaf(va[a].x, vb[b].x, inner[a][b]);
          inner[a][b] = fmaf(va[a].y, vb[b].y, inner[a][b]);
          inner[a][b] = fmaf(va[a].z, vb[b].z, inner[a][b]);
          inner[a][b] = fmaf(va[a].w, vb[b].w, inner[a][b]);
        }
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
    __syncthreads();   // the slot is refilled by the next iteration's copies
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
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

constexpr size_t kG32Smem = sizeof(float) * kG32Stages * 2 * kG32Slab;

template <class TX>
cudaError_t launch_trsm32_t(const TX *X, int64_t m, int64_t n, int64_t ldx, const float *Rf, const float *dinv,
                            const int32_t *perm, const int64_t *rank, float *Q, int64_t ldq, int NB,
                            cudaStream_t st) {
  const size_t smem = (size_t)NB * NB * 4 + (size_t)NB * 4;
#define RCQR_T32(NBV)                                                                                          \
  case NBV: {                                                                                                  \
    constexpr int RRV = NBV <= 64 ? 2 : 1;                                                                     \
    const unsigned blocks = (unsigned)((m + RRV * kT32Threads - 1) / (RRV * kT32Threads));                      \
    cudaError_t e = set_smem(trsm32_kernel<TX, NBV, RRV>, (int)smem);                                          \
    if (e != cudaSuccess) return e;                                                                            \
    trsm32_kernel<TX, NBV, RRV><<<blocks, kT32Threads, smem, st>>>(X, m, (int)n, ldx, Rf, dinv, perm, rank, Q, \
                                                                    ldq);                                      \
    break;                                                                                                     \
  }
  switch (NB) {
    RCQR_T32(16)
    RCQR_T32(32)
    RCQR_T32(48)
    RCQR_T32(64)
    default: return cudaErrorInvalidValue;
  }
#undef RCQR_T32
  return cudaGetLastError();
}

}  // namespace

bool trsm32_supported(int64_t n) { return n >= 1 && n <= 256; }

// R in FP32 for the substitution kernels: NB x NB, NB = n rounded up to 16 (row
// kernel) or to 64 (panel kernel, n > 64).
int trsm32_nb(int64_t n) { return n > 64 ? (int)((n + 63) / 64) * 64 : (int)((n + 15) / 16) * 16; }

size_t trsm32_workspace(int64_t n) {
  const int NB = trsm32_nb(n);
  Workspace w(nullptr, 0);
  w.take<float>((size_t)NB * NB);
  w.take<float>((size_t)NB);
  return w.used;
}

cudaError_t launch_trsm32(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, const double *R,
                          int64_t ldr, const int32_t *perm, const int64_t *rank, void *Q, int64_t ldq,
                          Workspace &ws, cudaStream_t st) {
  const int NB = trsm32_nb(n);
  float *Rf = ws.take<float>((size_t)NB * NB);
  float *dinv = ws.take<float>((size_t)NB);
  if (!Rf || !dinv) return cudaErrorMemoryAllocation;
  trsm32_prep_kernel<<<1, 256, 0, st>>>(R, (int)n, ldr, rank, NB, Rf, dinv);
  if (trsm_tcw_supported(n))   // 64 < n <= 128: blocked, off-diagonal products on the tensor cores
    return launch_trsm_tcw(X, m, n, ldx, prec, Rf, dinv, perm, rank, (float *)Q, ldq, nullptr, st);
  if (n > 64) {
    const unsigned blocks = (unsigned)((m + kT32Threads - 1) / kT32Threads);
    if (prec == RCQR_BF16)
      trsm32_wide_kernel<__nv_bfloat16><<<blocks, kT32Threads, 0, st>>>((const __nv_bfloat16 *)X, m, (int)n, ldx, Rf,
                                                                       NB, dinv, perm, rank, (float *)Q, ldq);
    else
      trsm32_wide_kernel<float><<<blocks, kT32Threads, 0, st>>>((const float *)X, m, (int)n, ldx, Rf, NB, dinv,
                                                               perm, rank, (float *)Q, ldq);
    return cudaGetLastError();
  }
  if (prec == RCQR_BF16)
    return launch_trsm32_t<__nv_bfloat16>((const __nv_bfloat16 *)X, m, n, ldx, Rf, dinv, perm, rank,
                                          (float *)Q, ldq, NB, st);
  return launch_trsm32_t<float>((const float *)X, m, n, ldx, Rf, dinv, perm, rank, (float *)Q, ldq, NB, st);
}

bool trsm32_gram_supported(int64_t n) { return n >= 1 && n <= 64; }

int trsm32_gram_groups(int64_t m) {
  const int64_t tiles = (m + kTGRows - 1) / kTGRows;
  return (int)std::max<int64_t>(1, std::min<int64_t>(2LL * num_sms(), tiles));
}

size_t trsm32_gram_workspace(int64_t m, int64_t n) {
  Workspace w(nullptr, 0);
  w.take<float>((size_t)64 * 64);
  w.take<float>((size_t)64);
  const int G = trsm_tc_supported(n) ? trsm_tc_gram_groups(m) : trsm32_gram_groups(m);
  w.take<double>((size_t)G * n * n);
  return w.used;
}

cudaError_t launch_trsm32_gram(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, const double *R,
                               int64_t ldr, const int32_t *perm, const int64_t *rank, float *Q, int64_t ldq,
                               double *A, int64_t lda, Workspace &ws, cudaStream_t st, int *dev_status) {
  const bool tc = trsm_tc_supported(n);
  const int NB = tc ? 64 : (int)((n + 15) / 16) * 16;
  float *Rf = ws.take<float>((size_t)64 * 64);
  float *dinv = ws.take<float>((size_t)64);
  const int G = tc ? trsm_tc_gram_groups(m) : trsm32_gram_groups(m);
  double *partial = ws.take<double>((size_t)G * n * n);
  if (!Rf || !dinv || !partial) return cudaErrorMemoryAllocation;
  trsm32_prep_kernel<<<1, 256, 0, st>>>(R, (int)n, ldr, rank, NB, Rf, dinv);
  if (tc) {
    cudaError_t e = launch_trsm_tc_gram(X, m, n, ldx, prec, Rf, dinv, perm, rank, Q, ldq, partial, dev_status, st);
    if (e != cudaSuccess) return e;
    return launch_gram_reduce(partial, G, n, A, lda, st);
  }
  const size_t smem = ((size_t)NB * NB + 64 + (size_t)64 * kTGStride) * sizeof(float);
  cudaError_t e = cudaSuccess;
#define RCQR_TG(NBV)                                                                                     \
  case NBV: {                                                                                            \
    if (prec == RCQR_BF16) {                                                                             \
      e = set_smem(trsm32_gram_kernel<__nv_bfloat16, NBV>, (int)smem);                                   \
      if (e != cudaSuccess) return e;                                                                    \
      trsm32_gram_kernel<__nv_bfloat16, NBV><<<G, kT32Threads, smem, st>>>(                              \
          (const __nv_bfloat16 *)X, m, (int)n, ldx, Rf, dinv, perm, rank, Q, ldq, partial);              \
    } else {                                                                                             \
      e = set_smem(trsm32_gram_kernel<float, NBV>, (int)smem);                                           \
      if (e != cudaSuccess) return e;                                                                    \
      trsm32_gram_kernel<float, NBV><<<G, kT32Threads, smem, st>>>((const float *)X, m, (int)n, ldx, Rf, \
                                                                   dinv, perm, rank, Q, ldq, partial);   \
    }                                                                                                    \
    break;                                                                                               \
  }
  switch (NB) {
    RCQR_TG(16)
    RCQR_TG(32)
    RCQR_TG(48)
    RCQR_TG(64)
    default: return cudaErrorInvalidValue;
  }
#undef RCQR_TG
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_gram_reduce(partial, G, n, A, lda, st);
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
  cudaError_t e = set_smem(gram32_kernel, (int)kG32Smem);
  if (e != cudaSuccess) return e;
  const int vec = ((uintptr_t)Q % 16 == 0) && (ldq % 4 == 0);
  gram32_kernel<<<grid, 256, kG32Smem, st>>>(Q, m, (int)n, ldq, rank, groups, partial, nullptr, 0, vec);
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
  cudaError_t e = set_smem(gram32_kernel, (int)kG32Smem);
  if (e != cudaSuccess) return e;
  const int vec = ((uintptr_t)A % 16 == 0) && (lda % 4 == 0) && ((uintptr_t)B % 16 == 0) && (ldb % 4 == 0);
  gram32_kernel<<<grid, 256, kG32Smem, st>>>(A, m, (int)n, lda, nullptr, groups, partial, B, ldb, vec);
  return cudaGetLastError();
}

}  // namespace rcqr
