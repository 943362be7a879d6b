// The second pass of RCholeskyQR2 on the mixed path, Q <- Q R'^{-1} (Alg. 3 step 4),
// as a product with the explicit inverse W = R'^{-1} on the tcgen05 tensor cores.
//
// R' is the Cholesky factor of the Gram matrix of the first pass's Q, which is well
// conditioned (Sec. 3.1), so cond(R') = cond(Q) = O(1) and Q W with W formed in FP64
// is as accurate as the substitution; the product has no dependency chain along the
// columns, so it maps onto whole-tile MMAs.
//
// Exactness of the leading term.  The tensor core's FP32 accumulation does not round
// to nearest, so its error does not average out over the rows of Q^T Q.  Every row t of
// a 128-row tile is therefore scaled by 2^(14 - e_t) (e_t = floor(log2 max |q|), so
// |a| < 2^15 for a = q 2^(14 - e_t)) and split into h = 256 rint(a / 256) (a digit of
// at most 8 bits times 256), m = RN_fp16(a - h) and l = RN_fp16(a - h - m), all exact
// FP16 operands; every column j of W the same way with its own e_j.  In the product of
// row t and column j every h_a h_b term is an integer below 2^14 times 2^16, so the
// K <= 128 term sum is exact in the FP32 accumulator D_hh whatever its rounding.  The
// seven next terms (h m, m h, h l, m m, l h, m l, l m; at most 2^-8 of the leading one)
// accumulate in a second accumulator D_s whose rounding errors are 2^-8 smaller; the
// dropped l l is below 2^-22 of |a||b|.  FP16 pieces carry 11 significant bits and the
// scale keeps l out of FP16's subnormal range for all but negligible entries, so every
// entry is represented to 2^-22 of itself and the whole product to about 2^-21 of
// |Q| |W| entrywise.  The result is (D_hh + D_s) 2^(e_t - 14) 2^(e_j - 14), rounded once.
//
// The Gram matrix A = Q^T Q of the first pass's Q (Alg. 3 step 2), 64 < n <= 128, uses
// the same pieces with the scales per tile and column (gram_tc_kernel below).
//
// Layout.  A CTA takes tiles of 128 rows (TMEM lane t = row t); NP = 64 or 128 padded
// columns.  The row pieces h | m | l form one K-major operand of K extent 3 NP (thread
// t writes its row's 8-column chunks as 16-byte core-matrix rows).  W is upper
// triangular, so K-step t (rows 16t .. 16t+15 of W) only reaches output columns >= 16t:
// its B operand holds just those NP - 16t columns (two K core matrices per 8-column
// group) and the MMA writes D columns 16t .. NP-1 (N = NP - 16t), half the work of the
// full product.
#include <algorithm>

#include <cuda_fp16.h>

#include "common.cuh"
#include "rcqr_internal.h"
#include "umma.cuh"

namespace rcqr {

namespace {

constexpr int kGR = 128;                        // rows per tile = TMEM lanes
constexpr uint32_t kGemmWaitRounds = 1u << 20;  // bounded waits: rounds of try_wait (<= 1 us each)

template <int NP>
struct GemmCfg {
  static constexpr int TPR = NP / 64;                       // threads per row (64 columns each)
  static constexpr int THREADS = kGR * TPR;
  static constexpr int KW = 3 * NP;                         // K extent of the row-piece operand
  static constexpr uint32_t YSBO = (KW / 8) * 128;          // its 8-row groups
  static constexpr int Y_BYTES = kGR * KW * 2;              // 48 KB / 96 KB
  static constexpr int W_PIECE = 32 * (NP * (NP / 16) - 16 * (NP / 16) * (NP / 16 - 1) / 2);  // triangle
  static constexpr int OFF_W = Y_BYTES;
  static constexpr int OFF_SC = OFF_W + 3 * W_PIECE;        // column scales 2^(e_j - 14) of W (NP floats)
  static constexpr int OFF_MX = OFF_SC + NP * 4;            // row maxima of the half rows (TPR x 128 words)
  static constexpr int SMEM = OFF_MX + TPR * kGR * 4;
  static constexpr uint32_t NCOLS = 4 * NP;                 // two tiles' D_hh | D_s
  static constexpr int CTAS = NP == 64 ? 2 : 1;
  static_assert(CTAS * (SMEM + 2048) <= 228 * 1024, "CTAS CTAs per SM");
  static_assert(CTAS * NCOLS <= 512, "TMEM");
};

// Byte offset of element (output column j, K row i) of one W piece in the triangular
// K-step regions: region t (i / 16 == t) holds columns j >= 16 t.
template <int NP>
__host__ __device__ constexpr uint32_t w_region(int t) {
  return 32u * (uint32_t)(NP * t - 16 * t * (t - 1) / 2);
}
template <int NP>
__host__ __device__ constexpr uint32_t w_offset(int j, int i) {
  const int t = i / 16;
  return w_region<NP>(t) + (uint32_t)((j - 16 * t) / 8) * 256u + (uint32_t)((i % 16) / 8) * 128u +
         (uint32_t)(j % 8) * 16u + (uint32_t)(i % 8) * 2u;
}

struct GemmArgs {
  float *Y;                   // m x n, ld ldy
  int64_t m;
  int n;
  int64_t ldy;
  const unsigned char *Wp;    // W's three pieces in their shared-memory layout, then 2^(e_j - 14) per column
  float *Z;                   // m x n, ld ldz; may be Y (each tile is read before it is written)
  int64_t ldz;
  int *status;                // nullable: RCQR_ETIMEOUT on a wait that gave up
};

__device__ __forceinline__ bool wait_mma(uint64_t *bar, uint32_t parity, int *fail) {
  for (uint32_t it = 0; it < kGemmWaitRounds; ++it) {
    if (*(volatile int *)fail) return false;
    if (umma::mbar_try_wait_hint(bar, parity, 1000)) return true;
  }
  *(volatile int *)fail = 1;
  return false;
}

// The scale pair 2^(14-e), 2^(e-14) of a row (or column) whose largest magnitude has
// the FP32 biased exponent be; (0, 0) for a zero row or one below 2^-112, which is then
// taken as zero.
__device__ __forceinline__ void fixed_scales(int be, float &sc, float &isc) {
  const bool ok = be >= 15 && be <= 250;
  sc = ok ? __uint_as_float((uint32_t)(127 + 141 - be) << 23) : 0.0f;
  isc = ok ? __uint_as_float((uint32_t)(be - 14) << 23) : 0.0f;
}

// h, m, l of two scaled values a0, a1 (|a| < 2^15) as FP16 pairs: h = 256 rint(a / 256)
// exact, m = RN(a - h), l = RN(a - h - m); the differences are exact in FP32.
__device__ __forceinline__ void split_row2(float a0, float a1, uint32_t &h, uint32_t &mm, uint32_t &l) {
  const float h0 = rintf(a0 * 0x1p-8f) * 256.0f, h1 = rintf(a1 * 0x1p-8f) * 256.0f;
  const __half2 hb = __floats2half2_rn(h0, h1);
  const float r0 = a0 - h0, r1 = a1 - h1;
  const __half2 mb = __floats2half2_rn(r0, r1);
  const float2 mf = __half22float2(mb);
  const __half2 lb = __floats2half2_rn(r0 - mf.x, r1 - mf.y);
  h = *reinterpret_cast<const uint32_t *>(&hb);
  mm = *reinterpret_cast<const uint32_t *>(&mb);
  l = *reinterpret_cast<const uint32_t *>(&lb);
}

template <int NP>
__global__ void __launch_bounds__(GemmCfg<NP>::THREADS, GemmCfg<NP>::CTAS) gemm_tc_kernel(GemmArgs a) {
  using C = GemmCfg<NP>;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *Ys = smem;
  unsigned char *Ws = smem + C::OFF_W;
  float *Isw = reinterpret_cast<float *>(smem + C::OFF_SC);
  unsigned *Mx = reinterpret_cast<unsigned *>(smem + C::OFF_MX);
  __shared__ uint64_t bar_mma, bar_drain;
  __shared__ uint32_t tslot;
  __shared__ int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5;
  const int trow = tid % kGR, half = tid / kGR;        // this thread's row and its 64-column half
  const int n = a.n;

  // ---- set-up: W's pieces and column scales (prepared once by tri_inv_split_kernel)
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(a.Wp);
    uint4 *dst = reinterpret_cast<uint4 *>(Ws);
    for (int e = tid; e < 3 * C::W_PIECE / 16; e += C::THREADS) dst[e] = src[e];
    const float *isw = reinterpret_cast<const float *>(a.Wp + 3 * C::W_PIECE);
    for (int j = tid; j < NP; j += C::THREADS) Isw[j] = isw[j];
  }
  if (tid == 0) {
    umma::mbar_init(&bar_mma, 1);
    umma::mbar_init(&bar_drain, 1);
    s_fail = 0;
  }
  if (warp == 0) umma::tmem_alloc(&tslot, C::NCOLS);
  umma::fence_proxy_async();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tbase = tslot;
  const uint32_t lane_base = tbase + ((uint32_t)(32 * (warp & 3)) << 16);
  const uint32_t ys_addr = umma::smem_u32(Ys), ws_addr = umma::smem_u32(Ws);
  const uint32_t row_sw = (uint32_t)(trow / 8) * C::YSBO + (uint32_t)(trow % 8) * 16;
  uint32_t ph = 0;

  const int64_t tiles = (a.m + kGR - 1) / kGR;
  // this thread's 64 values of its row; the next tile's are loaded while the current
  // tile's MMAs run and its results are written
  float y[64];
  auto load_tile = [&](int64_t tl) {
    const int64_t rw = tl * kGR + trow;
    const bool lv = tl < tiles && rw < a.m;
#pragma unroll
    for (int c = 0; c < 64; ++c) {
      const int j = 64 * half + c;
      y[c] = (lv && j < n) ? a.Y[rw + (int64_t)j * a.ldy] : 0.0f;
    }
  };
  // Z = (D_hh + D_s) 2^(e_t - 14) 2^(e_j - 14) of a finished tile, this thread's row and half
  auto readback = [&](uint32_t dbase, int64_t rw, bool lv, float rsc) {
    int64_t ldz = a.ldz;
    asm volatile("" : "+l"(ldz));
#pragma unroll
    for (int c16 = 0; c16 < 4; ++c16) {
      uint32_t vh[16], vs[16];
      const uint32_t col = (uint32_t)(64 * half + 16 * c16);
      umma::tmem_ld16(lane_base + dbase + col, vh);
      umma::tmem_ld16(lane_base + dbase + NP + col, vs);
      umma::tmem_wait_ld();
      if (lv) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int j = (int)col + u;
          if (j < n) a.Z[rw + (int64_t)j * ldz] = (__uint_as_float(vh[u]) + __uint_as_float(vs[u])) * rsc * Isw[j];
        }
      }
    }
  };
  // software pipeline: the MMAs of tile k (TMEM buffer k % 2) run while tile k - 1's
  // results are read back from the other buffer
  load_tile(blockIdx.x);
  uint32_t buf = 0;
  bool have_prev = false, prev_live = false;
  int64_t prev_row = 0;
  float prev_isc = 0.0f;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t row = tile * kGR + trow;
    const bool live = row < a.m;
    unsigned mx = 0;
#pragma unroll
    for (int c = 0; c < 64; ++c) mx = max(mx, __float_as_uint(y[c]) & 0x7FFFFFFFu);
    if constexpr (C::TPR > 1) {
      Mx[half * kGR + trow] = mx;
      __syncthreads();
      mx = max(Mx[trow], Mx[kGR + trow]);
    }
    float sc, isc;                                     // the row's scale pair
    fixed_scales((int)(mx >> 23), sc, isc);
    // the row pieces, K-major (piece p occupies K columns p NP .. p NP + NP - 1); the
    // previous tile's MMAs, their last readers, completed in the previous iteration
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8) {
      uint32_t hw[4], mw[4], lw[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) split_row2(y[8 * c8 + 2 * p] * sc, y[8 * c8 + 2 * p + 1] * sc, hw[p], mw[p], lw[p]);
      const int col = 64 * half + 8 * c8;
      *reinterpret_cast<uint4 *>(Ys + row_sw + ((0 * NP + col) / 8) * 128) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint4 *>(Ys + row_sw + ((1 * NP + col) / 8) * 128) = make_uint4(mw[0], mw[1], mw[2], mw[3]);
      *reinterpret_cast<uint4 *>(Ys + row_sw + ((2 * NP + col) / 8) * 128) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
    load_tile(tile + gridDim.x);
    umma::fence_proxy_async();
    umma::fence_before_sync();
    __syncthreads();   // the pieces written; the previous read-back of this TMEM buffer done
    if (tid == 0 && !*(volatile int *)&s_fail) {
      umma::fence_after_sync();
      // (row piece, W piece) of the leading product and of the seven next ones
      const int pa[8] = {0, 0, 1, 0, 1, 2, 1, 2}, pw[8] = {0, 1, 0, 2, 1, 0, 2, 1};
      const uint32_t dbuf = tbase + buf * (2u * NP);
#pragma unroll
      for (int t = 0; t < NP / 16; ++t) {
        const int N = NP - 16 * t;
        const uint32_t id = umma::idesc_f16_f32(kGR, N);
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          const uint64_t ad = umma::smem_desc(ys_addr + ((pa[p] * NP + 16 * t) / 8) * 128, 128, C::YSBO);
          const uint64_t bd = umma::smem_desc(ws_addr + pw[p] * C::W_PIECE + w_region<NP>(t), 128, 256);
          const uint32_t d = dbuf + (p == 0 ? 0u : (uint32_t)NP) + 16u * t;
          const bool first = t == 0 && (p == 0 || p == 1);
          umma::mma_bf16(d, ad, bd, id, first ? 0u : 1u);
        }
      }
      umma::mma_commit(&bar_mma);
    }
    if (have_prev) {
      umma::fence_after_sync();
      readback((buf ^ 1u) * (2u * NP), prev_row, prev_live, prev_isc);
    }
    wait_mma(&bar_mma, ph, &s_fail);
    ph ^= 1u;
    umma::fence_before_sync();
    have_prev = true;
    prev_row = row;
    prev_live = live;
    prev_isc = isc;
    buf ^= 1u;
  }
  if (have_prev) {
    umma::fence_after_sync();
    readback((buf ^ 1u) * (2u * NP), prev_row, prev_live, prev_isc);
  }

  // drain: every MMA issued by thread 0 has finished before TMEM is released
  if (tid == 0) {
    umma::mma_commit(&bar_drain);
    if (!umma::mbar_wait(&bar_drain, 0u, 1u << 22)) s_fail = 1;
  }
  umma::fence_before_sync();
  __syncthreads();
  if (tid == 0 && *(volatile int *)&s_fail && a.status && atomicCAS(a.status, 0, (int)RCQR_ETIMEOUT) == 0)
    a.status[1] = -1;
  if (warp == 0) umma::tmem_dealloc(tbase, C::NCOLS);
}

// ---------------------------------------------------------------------------------
// A = Q^T Q for 64 < n <= 128 (NP = 128), FP32 Q.  A CTA of 512 threads takes tiles of
// 128 rows; thread (r, g) holds row r of the tile and columns 32 g .. 32 g + 31, and in
// the fold it owns row i = r of A at the same columns (TMEM lane i, warp w reading lanes
// 32 (w % 4) ..).  Per tile and column j, the column is scaled by 2^(14 - e_j) (e_j from
// the tile's largest |q|) and split into h (8-bit digit times 256), m, l as FP16, K-major
// along the columns like gemm_tc_kernel's row pieces, which the tensor cores read as the
// transposed (MN-major) operands.  Every h_ri h_rj is an integer below 2^14 times 2^16,
// so D_hh = H^T H over the 128 rows is exact; H^T M (8 accumulations, at most 2^-7 of
// the leading term), H^T L and M^T M go to accumulators of their own.  After every tile
// each thread adds
//     (h h / 2 + h m + h l + m m / 2) 2^(e_i - 14) 2^(e_j - 14)
// for its 32 entries into FP32 Kahan sums S; the CTA's partial is S in FP64, and the
// reduction forms A = sum over CTAs of (S + S^T) (the dropped m l, l m, l l are below
// 2^-26 of |q_i||q_j|).
constexpr int kGramThreads = 512;
constexpr int kGramCols = 32;                 // columns per thread
constexpr int kGramNP = 128;
constexpr uint32_t kGramYSBO = (3 * kGramNP / 8) * 128;
constexpr int kGramY = kGR * 3 * kGramNP * 2;  // 96 KB of pieces
constexpr int kGramRaw = kGR * kGramNP * 4;      // one raw tile, column-major, 64 KB
constexpr int kGramSmem = kGramRaw + kGramY + 4 * kGramNP * 4 + 2 * kGramNP * 4;   // raw, pieces, maxima, scales

__device__ __forceinline__ void cp_async16z(void *dst, const void *src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(umma::smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit_all() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Copies tile `tile` of Q (128 rows x n columns) into the raw buffer, column c at floats
// c * 128 .. (rows past m read as zero): asynchronously in 16-byte pieces when Q's rows
// are 16-byte aligned (vec), else by plain loads.
__device__ __forceinline__ void gram_fetch_tile(const float *__restrict__ Q, int64_t m, int n, int64_t ldq,
                                                int64_t tile, float *raw, bool vec) {
  const int64_t r0 = tile * kGR;
  for (int e = threadIdx.x; e < kGramNP * (kGR / 4); e += kGramThreads) {
    const int c = e / (kGR / 4), q4 = e % (kGR / 4);
    if (c >= n) continue;
    const int64_t row = r0 + 4 * q4;
    const int64_t left = m - row;
    const int valid = left > 0 ? (int)(left < 4 ? left : 4) : 0;
    float *dst = raw + c * kGR + 4 * q4;
    if (vec) {
      cp_async16z(dst, valid > 0 ? Q + row + (int64_t)c * ldq : Q, 4 * valid);
    } else {
      float v[4];
#pragma unroll
      for (int k4 = 0; k4 < 4; ++k4) v[k4] = k4 < valid ? Q[row + k4 + (int64_t)c * ldq] : 0.0f;
      *reinterpret_cast<float4 *>(dst) = make_float4(v[0], v[1], v[2], v[3]);
    }
  }
  cp_async_commit_all();
}

__global__ void __launch_bounds__(kGramThreads, 1) gram_tc_kernel(const float *__restrict__ Q, int64_t m, int n,
                                                                 int64_t ldq, double *partial, int *status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  float *raw = reinterpret_cast<float *>(smem);
  unsigned char *Ys = smem + kGramRaw;
  unsigned *Wmax = reinterpret_cast<unsigned *>(smem + kGramRaw + kGramY);      // 4 x NP: per warp row group
  float *Sc = reinterpret_cast<float *>(smem + kGramRaw + kGramY + 4 * kGramNP * 4), *Isc = Sc + kGramNP;
  __shared__ uint64_t bar_mma, bar_drain;
  __shared__ uint32_t tslot;
  __shared__ int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int trow = tid % kGR, grp = tid / kGR;          // row of the tile, column group
  const int c0 = kGramCols * grp;
  const bool vec = ((uintptr_t)Q % 16 == 0) && (ldq % 4 == 0);
  if (tid == 0) {
    umma::mbar_init(&bar_mma, 1);
    umma::mbar_init(&bar_drain, 1);
    s_fail = 0;
  }
  if (warp == 0) umma::tmem_alloc(&tslot, 512u);        // D_hh | D_hm | D_hl | D_mm, 128 columns each
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tbase = tslot;
  const uint32_t lane_base = tbase + ((uint32_t)(32 * (warp & 3)) << 16);
  const uint32_t ys_addr = umma::smem_u32(Ys);
  const uint32_t row_sw = (uint32_t)(trow / 8) * kGramYSBO + (uint32_t)(trow % 8) * 16;
  float acc[kGramCols], cmp[kGramCols];
#pragma unroll
  for (int c = 0; c < kGramCols; ++c) acc[c] = cmp[c] = 0.0f;
  uint32_t ph = 0;

  // per tile: split the raw tile (copied during the previous tile's MMAs and fold),
  // start the copy of the next tile, run the MMAs, fold
  const int64_t tiles = (m + kGR - 1) / kGR;
  if ((int64_t)blockIdx.x < tiles) gram_fetch_tile(Q, m, n, ldq, blockIdx.x, raw, vec);
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t row = tile * kGR + trow;
    const bool live = row < m;
    cp_async_wait_all();
    __syncthreads();                                    // the raw tile is complete
    float y[kGramCols];
#pragma unroll
    for (int c = 0; c < kGramCols; ++c) y[c] = (live && c0 + c < n) ? raw[(c0 + c) * kGR + trow] : 0.0f;
    // per column, the tile's largest |q|: warp maxima, then the four row groups
#pragma unroll
    for (int c = 0; c < kGramCols; ++c) {
      const unsigned mx = __reduce_max_sync(0xffffffffu, __float_as_uint(y[c]) & 0x7FFFFFFFu);
      if (lane == 0) Wmax[(warp & 3) * kGramNP + c0 + c] = mx;
    }
    __syncthreads();
    if (tid < kGramNP) {
      const unsigned mx = max(max(Wmax[tid], Wmax[kGramNP + tid]), max(Wmax[2 * kGramNP + tid], Wmax[3 * kGramNP + tid]));
      fixed_scales((int)(mx >> 23), Sc[tid], Isc[tid]);
    }
    __syncthreads();
#pragma unroll
    for (int c8 = 0; c8 < kGramCols / 8; ++c8) {
      uint32_t hw[4], mw[4], lw[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int c = 8 * c8 + 2 * p;
        split_row2(y[c] * Sc[c0 + c], y[c + 1] * Sc[c0 + c + 1], hw[p], mw[p], lw[p]);
      }
      const int col = c0 + 8 * c8;
      *reinterpret_cast<uint4 *>(Ys + row_sw + ((0 * kGramNP + col) / 8) * 128) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint4 *>(Ys + row_sw + ((1 * kGramNP + col) / 8) * 128) = make_uint4(mw[0], mw[1], mw[2], mw[3]);
      *reinterpret_cast<uint4 *>(Ys + row_sw + ((2 * kGramNP + col) / 8) * 128) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
    umma::fence_proxy_async();
    umma::fence_before_sync();
    __syncthreads();                                    // pieces written; the raw buffer is free
    if (tid == 0 && !*(volatile int *)&s_fail) {
      umma::fence_after_sync();
      // MN-major views: 8-column groups 128 B apart (SBO), 8-row groups kGramYSBO apart
      // (LBO); per K-step H^T [H | M] (N = 256: the H and M pieces are adjacent),
      // H^T L, M^T M
      const uint32_t id256 = umma::idesc_f16_f32(kGR, 2 * kGramNP) | (1u << 15) | (1u << 16);
      const uint32_t id128 = umma::idesc_f16_f32(kGR, kGramNP) | (1u << 15) | (1u << 16);
#pragma unroll
      for (int t = 0; t < kGR / 16; ++t) {
        const uint32_t kofs = (uint32_t)(2 * t) * kGramYSBO;
        const uint64_t dh = umma::smem_desc(ys_addr + kofs, kGramYSBO, 128);
        const uint64_t dm = umma::smem_desc(ys_addr + kofs + (kGramNP / 8) * 128, kGramYSBO, 128);
        const uint64_t dl = umma::smem_desc(ys_addr + kofs + (2 * kGramNP / 8) * 128, kGramYSBO, 128);
        const uint32_t acc_flag = t > 0 ? 1u : 0u;
        umma::mma_bf16(tbase, dh, dh, id256, acc_flag);                    // hh | hm
        umma::mma_bf16(tbase + 2 * kGramNP, dh, dl, id128, acc_flag);      // hl
        umma::mma_bf16(tbase + 3 * kGramNP, dm, dm, id128, acc_flag);      // mm
      }
      umma::mma_commit(&bar_mma);
    }
    if (tile + gridDim.x < tiles) gram_fetch_tile(Q, m, n, ldq, tile + gridDim.x, raw, vec);
    wait_mma(&bar_mma, ph, &s_fail);
    ph ^= 1u;
    umma::fence_after_sync();
    // fold: row i = trow of this tile's A, columns c0 ..
    const float isi = Isc[trow];
#pragma unroll
    for (int c8 = 0; c8 < kGramCols / 8; ++c8) {
      uint32_t vhh[8], vhm[8], vhl[8], vmm[8];
      const uint32_t col = (uint32_t)(c0 + 8 * c8);
      umma::tmem_ld8(lane_base + col, vhh);
      umma::tmem_ld8(lane_base + kGramNP + col, vhm);
      umma::tmem_ld8(lane_base + 2 * kGramNP + col, vhl);
      umma::tmem_ld8(lane_base + 3 * kGramNP + col, vmm);
      umma::tmem_wait_ld();
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int c = 8 * c8 + u;
        const float t = (0.5f * (__uint_as_float(vhh[u]) + __uint_as_float(vmm[u])) + __uint_as_float(vhm[u]) +
                         __uint_as_float(vhl[u])) * (isi * Isc[c0 + c]);
        const float yk = t - cmp[c];
        const float sk = acc[c] + yk;
        cmp[c] = (sk - acc[c]) - yk;
        acc[c] = sk;
      }
    }
    umma::fence_before_sync();
    __syncthreads();   // TMEM, the pieces and the scales are free for the next tile
  }
  cp_async_wait_all();
  // the CTA's partial S (row i = trow, this thread's columns), in FP64
  const bool failed = *(volatile int *)&s_fail != 0;
  if (trow < n) {
    double *pb = partial + (int64_t)blockIdx.x * n * n;
#pragma unroll
    for (int c = 0; c < kGramCols; ++c) {
      const int j = c0 + c;
      if (j < n) pb[trow + (int64_t)j * n] = failed ? __longlong_as_double(0x7FF8000000000000ll)
                                                    : (double)acc[c] - (double)cmp[c];
    }
  }
  if (tid == 0) {
    umma::mma_commit(&bar_drain);
    if (!umma::mbar_wait(&bar_drain, 0u, 1u << 22)) s_fail = 1;
  }
  umma::fence_before_sync();
  __syncthreads();
  if (tid == 0 && *(volatile int *)&s_fail && status && atomicCAS(status, 0, (int)RCQR_ETIMEOUT) == 0) status[1] = -1;
  if (warp == 0) umma::tmem_dealloc(tbase, 512u);
}

// A(i, j) = sum over the CTAs g of S_g(i, j) + S_g(j, i), in a fixed order (one warp per entry).
__global__ void gram_sym_reduce_kernel(const double *__restrict__ partial, int groups, int n, double *__restrict__ A,
                                       int64_t lda) {
  const int64_t idx = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (idx >= (int64_t)n * n) return;
  const int i = (int)(idx % n), j = (int)(idx / n);
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int g = lane; g < groups; g += 32) {
    const double *pg = partial + (int64_t)g * n * n;
    s += pg[i + (int64_t)j * n] + pg[j + (int64_t)i * n];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) A[i + (int64_t)j * lda] = s;
}

int gram_tc_groups(int64_t m) {
  const int64_t tiles = (m + kGR - 1) / kGR;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, num_sms()));
}

// W = R'^{-1} on the leading r x r block (zero elsewhere), then W's pieces for
// gemm_tc_kernel: one warp per column c of the padded NP columns.  Back substitution
// w_i = -(sum_{l = i+1..c} R'_il w_l) / R'_ii (w_c = 1 / R'_cc), the sum split over the
// lanes, R' staged in shared memory row by row with the reciprocals of its diagonal;
// then the column's scale 2^(14 - e_c) from its largest |w|, and h = 256 rint(b / 256),
// m = RN_fp16(b - h), l = RN_fp16(b - h - m) of b = w 2^(14 - e_c), written in the
// triangular layout of gemm_tc_kernel's shared memory (rows i <= 16 (c / 16) + 15).
constexpr int kInvWarps = 8;
template <int NP>
__global__ void __launch_bounds__(32 * kInvWarps) tri_inv_split_kernel(const double *__restrict__ Rp, int n,
                                                                       int64_t ldrp, const int64_t *rank,
                                                                       unsigned char *Wp) {
  using C = GemmCfg<NP>;
  extern __shared__ double inv_smem[];
  double *Rs = inv_smem;                                 // n x n, row-major: Rs[i * n + l]
  double *rd = Rs + (size_t)n * n;                       // 1 / R'_ii
  double *ws = rd + n;                                   // one column per warp (NP entries)
  const int r = rank ? (int)(*rank < (int64_t)n ? *rank : (int64_t)n) : n;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, l = e / n;
    Rs[i * n + l] = Rp[i + (int64_t)l * ldrp];
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) rd[i] = 1.0 / Rp[i + (int64_t)i * ldrp];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * kInvWarps + warp;
  if (c >= NP) return;
  double *w = ws + (size_t)warp * NP;
  for (int i = lane; i < NP; i += 32) w[i] = 0.0;
  __syncwarp();
  if (c < r) {
    if (lane == 0) w[c] = rd[c];
    __syncwarp();
    for (int i = c - 1; i >= 0; --i) {
      double s = 0.0;
      for (int l = i + 1 + lane; l <= c; l += 32) s = fma(Rs[i * n + l], w[l], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) w[i] = -s * rd[i];
      __syncwarp();
    }
  }
  double mx = 0.0;
  for (int i = lane; i <= c; i += 32) mx = fmax(mx, fabs(w[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  // e = floor(log2 mx) from the FP32 rounding of mx (one binade high at most, which
  // keeps |b| < 2^15); zero or out-of-range columns get the scale 0
  const int be = (int)(__float_as_uint((float)mx) >> 23);
  const bool ok = be >= 15 && be <= 250;
  const float sc = ok ? __uint_as_float((uint32_t)(127 + 141 - be) << 23) : 0.0f;
  const float isc = ok ? __uint_as_float((uint32_t)(be - 14) << 23) : 0.0f;
  const int iend = 16 * (c / 16) + 16;                   // rows of the column in the triangular regions
  for (int i = lane; i < iend; i += 32) {
    const double b = w[i] * (double)sc;
    const double h = 256.0 * rint(b * 0x1p-8);
    const __half mb = __double2half(b - h);
    const __half lb = __double2half(b - h - (double)__half2float(mb));
    const uint32_t off = w_offset<NP>(c, i);
    *reinterpret_cast<__half *>(Wp + off) = __float2half_rn((float)h);
    *reinterpret_cast<__half *>(Wp + C::W_PIECE + off) = mb;
    *reinterpret_cast<__half *>(Wp + 2 * C::W_PIECE + off) = lb;
  }
  if (lane == 0) reinterpret_cast<float *>(Wp + 3 * C::W_PIECE)[c] = isc;
}

template <int NP>
int gemm_grid(int64_t m) {
  const int64_t tiles = (m + kGR - 1) / kGR;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)GemmCfg<NP>::CTAS * num_sms()));
}

template <int NP>
cudaError_t launch_gemm(const GemmArgs &a, cudaStream_t st) {
  auto kern = gemm_tc_kernel<NP>;
  cudaError_t e = set_smem(kern, GemmCfg<NP>::SMEM);
  if (e != cudaSuccess) return e;
  kern<<<gemm_grid<NP>(a.m), GemmCfg<NP>::THREADS, GemmCfg<NP>::SMEM, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

bool gemm_tc_supported(int64_t n) { return n > 64 && n <= 128; }

bool gram_tc_supported(int64_t n) { return n > 64 && n <= 128; }

size_t gram_tc_workspace(int64_t m, int64_t n) {
  Workspace w(nullptr, 0);
  w.take<double>((size_t)gram_tc_groups(m) * n * n);
  return w.used;
}

cudaError_t launch_gram_tc(const float *Q, int64_t m, int64_t n, int64_t ldq, double *A, int64_t lda, int *status,
                           Workspace &ws, cudaStream_t st) {
  const int G = gram_tc_groups(m);
  double *partial = ws.take<double>((size_t)G * n * n);
  if (!partial) return cudaErrorMemoryAllocation;
  cudaError_t e = set_smem(gram_tc_kernel, kGramSmem);
  if (e != cudaSuccess) return e;
  gram_tc_kernel<<<G, kGramThreads, kGramSmem, st>>>(Q, m, (int)n, ldq, partial, status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  gram_sym_reduce_kernel<<<(unsigned)((n * n * 32 + 255) / 256), 256, 0, st>>>(partial, G, (int)n, A, lda);
  return cudaGetLastError();
}

size_t gemm_tc_workspace(int64_t n) {
  Workspace w(nullptr, 0);
  w.take<unsigned char>(n <= 64 ? 3 * GemmCfg<64>::W_PIECE + 64 * 4 : 3 * GemmCfg<128>::W_PIECE + 128 * 4);
  return w.used;
}

template <int NP>
cudaError_t inverse_times(float *Q, int64_t m, int64_t n, int64_t ldq, const double *Rp, int64_t ldrp,
                          const int64_t *rank, int *status, Workspace &ws, cudaStream_t st) {
  unsigned char *Wp = ws.take<unsigned char>(3 * GemmCfg<NP>::W_PIECE + NP * 4);
  if (!Wp) return cudaErrorMemoryAllocation;
  const size_t inv_smem = ((size_t)n * n + n + (size_t)kInvWarps * NP) * sizeof(double);
  cudaError_t e = set_smem(tri_inv_split_kernel<NP>, (int)inv_smem);
  if (e != cudaSuccess) return e;
  tri_inv_split_kernel<NP><<<NP / kInvWarps, 32 * kInvWarps, inv_smem, st>>>(Rp, (int)n, ldrp, rank, Wp);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  GemmArgs a{Q, m, (int)n, ldq, Wp, Q, ldq, status};
  return launch_gemm<NP>(a, st);
}

cudaError_t launch_inverse_times(float *Q, int64_t m, int64_t n, int64_t ldq, const double *Rp, int64_t ldrp,
                                 const int64_t *rank, int *status, Workspace &ws, cudaStream_t st) {
  return n <= 64 ? inverse_times<64>(Q, m, n, ldq, Rp, ldrp, rank, status, ws, st)
                 : inverse_times<128>(Q, m, n, ldq, Rp, ldrp, rank, status, ws, st);
}

}  // namespace rcqr
