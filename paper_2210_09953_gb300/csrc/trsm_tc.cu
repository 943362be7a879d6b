// Q = X R^{-1} (Alg. 2 step 3) for 32 < n <= 64 as a blocked substitution on
// the tcgen05 tensor cores, fused with the Gram matrix A = Q^T Q of the second
// pass (Alg. 3 step 2): the first pass of RCholeskyQR2 on the mixed path.
// (The template keeps GRAM = false, the substitution alone; the library uses the
// FP32 SIMT substitution there, which measured faster on its own.)
//
// A CTA of 128 threads takes tiles of 128 rows (thread t owns row t of the tile
// and TMEM lane t; two or three CTAs per SM hide each other's latencies).  The
// 64 (padded) columns form four blocks
// of 16.  For block J the thread forms y_J = x_J - (sum_{I<J} q_I R_{I,J}) and
// solves the 16 x 16 triangular system y_J = q_J R_{J,J} by substitution in
// FP32 registers (the diagonal block is never inverted).  The off-diagonal
// products run on the tensor cores, right-looking: once block J is solved, its
// q_J is split exactly into three bf16 pieces q = h + m + l (8 significant bits
// each, RN: the sum is exact for an FP32 q), and one group of MMAs adds
// q_J R_{J,>J} into the FP32 TMEM accumulator of the later columns.  R (rounded
// to FP32 once) is split the same way; the six products with piece indices
// summing to at most two are kept (the dropped ones are below 2^-26 of
// |q||R|), so each update carries the error of an FP32 sum of products, and
// the row-wise backward error stays that of the FP32 substitution,
// Q (R + dR) = X with |dR| <= c n u |R|, u = 2^-24 (Higham Thm. 8.5).
//
// The Gram (GRAM = true) is formed from a second split of the finished rows,
// read by the tensor cores as the transposed (MN-major) operand: per tile and
// column c, h = an 8-bit fixed-point digit of q relative to the column's largest
// |q| in the tile (h = round(q 2^(6-e)) 2^(e-6), e = floor(log2 max |q|)), then
// m = RN_bf16(q - h), l = RN_bf16(q - h - m).  Every h_i h_j is an integer
// multiple of 2^(e_i + e_j - 12) below 2^14 of them, so the 128-row sums of the
// leading term (h,h) are exact in the FP32 accumulator whatever its rounding;
// the other terms are at most 2^-8 of it.  Per tile, A = [h; m]^T times
// B = [h | m] gives (h,h) + (h,m) in lanes 0..63 and (m,h) + (m,m) in lanes
// 64..127, folded into per-thread FP32 Kahan sums; [h; m]^T l (2^-16 of the
// leading term) accumulates in TMEM across the tiles and its transpose supplies
// l^T h and l^T m.  The per-CTA partials go to FP64 and are summed in a fixed
// order by the Gram reduction.
#include <algorithm>

#include "common.cuh"
#include "rcqr_internal.h"
#include "umma.cuh"

namespace rcqr {

namespace {

constexpr int kTR = 128;            // rows per tile = TMEM lanes = threads per CTA
constexpr int kTN = 64;             // padded columns (four blocks of 16)
constexpr int kRSlice = kTN * kTN * 2;          // one bf16 slice of R: 8 KiB
constexpr uint32_t kRSBO = (kTN / 8) * 128;     // R slice: 8-column groups 1 KiB apart
constexpr uint32_t kWaitRounds = 1u << 20;      // bounded waits: rounds of try_wait (<= 1 us each)

template <bool GRAM>
struct TcCfg {
  static constexpr int CW = GRAM ? 64 : 48;         // columns of one piece in the slice buffer
  static constexpr int QW = 3 * CW;                  // h | m | l
  static constexpr uint32_t QSBO = (QW / 8) * 128;   // 8-row groups of the slice buffer
  static constexpr int Q_BYTES = kTR * QW * 2;
  static constexpr uint32_t NCOLS = GRAM ? 256u : 64u;   // TMEM: update acc (48) [+ P 128 + L 64]
  static constexpr uint32_t P_COL = 64;
  static constexpr uint32_t L_COL = 192;
  // byte offsets of the dynamic shared memory
  static constexpr int OFF_R = Q_BYTES;                   // 3 R pieces
  static constexpr int OFF_RD = OFF_R + 3 * kRSlice;      // diagonal blocks, 4 x 16 x 16 floats
  static constexpr int OFF_DS = OFF_RD + 4 * 256 * 4;     // dinv, Sc, Isc: 3 x 64 floats
  static constexpr int OFF_WMAX = OFF_DS + 3 * 64 * 4;    // per-warp column maxima: 4 x 64 words
  static constexpr int OFF_SRC = OFF_WMAX + 4 * 64 * 4;   // source columns: 64 ints
  static constexpr int SMEM = OFF_SRC + 64 * 4;
  static constexpr int CTAS = GRAM ? 2 : 3;               // per SM (TMEM, registers, shared memory)
  static_assert(CTAS * (SMEM + 2048) <= 228 * 1024, "CTAS CTAs per SM");
};

struct TcTrsmArgs {
  const void *X;
  int64_t m;
  int n;
  int64_t ldx;
  const float *Rf;      // 64 x 64 FP32, column-major, zero beyond the rank (trsm32_prep_kernel)
  const float *dinv;    // fl32(1 / R_jj), 0 beyond the rank
  const int32_t *perm;  // nullable
  const int64_t *rank;  // nullable
  float *Q;
  int64_t ldq;
  double *partial;      // GRAM: one n x n FP64 partial per CTA
  int *status;          // nullable: RCQR_ETIMEOUT on a wait that gave up
};

__device__ __forceinline__ float to_f32v(float x) { return x; }
__device__ __forceinline__ float to_f32v(__nv_bfloat16 x) { return __bfloat162float(x); }

// Exact three-way bf16 split of two FP32 values: x = h + m + l for each.
__device__ __forceinline__ void split3(float x0, float x1, uint32_t &h, uint32_t &mm, uint32_t &l) {
  const __nv_bfloat162 hb = __floats2bfloat162_rn(x0, x1);
  const float2 hf = __bfloat1622float2(hb);
  const float r0 = x0 - hf.x, r1 = x1 - hf.y;
  const __nv_bfloat162 mb = __floats2bfloat162_rn(r0, r1);
  const float2 mf = __bfloat1622float2(mb);
  const __nv_bfloat162 lb = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
  h = *reinterpret_cast<const uint32_t *>(&hb);
  mm = *reinterpret_cast<const uint32_t *>(&mb);
  l = *reinterpret_cast<const uint32_t *>(&lb);
}

// The Gram split of two FP32 values: h = round(x sc) isc (an exact fixed-point digit,
// sc = 2^(6-e), isc = 2^(e-6), or 0 when sc = 0), then m and l as in split3.
__device__ __forceinline__ void split_fixed(float x0, float x1, float sc0, float sc1, float isc0, float isc1,
                                            uint32_t &h, uint32_t &mm, uint32_t &l) {
  const float h0 = rintf(x0 * sc0) * isc0, h1 = rintf(x1 * sc1) * isc1;
  const __nv_bfloat162 hb = __floats2bfloat162_rn(h0, h1);     // exact: at most 8 significant bits
  const float r0 = x0 - h0, r1 = x1 - h1;
  const __nv_bfloat162 mb = __floats2bfloat162_rn(r0, r1);
  const float2 mf = __bfloat1622float2(mb);
  const __nv_bfloat162 lb = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
  h = *reinterpret_cast<const uint32_t *>(&hb);
  mm = *reinterpret_cast<const uint32_t *>(&mb);
  l = *reinterpret_cast<const uint32_t *>(&lb);
}

// tcgen05 instruction descriptor, kind::f16, BF16 x BF16 -> FP32, both operands MN-major.
__host__ __device__ constexpr uint32_t idesc_bf16_f32_mn(int M, int N) {
  return umma::idesc_bf16_f32(M, N) | (1u << 15) | (1u << 16);
}

// Bounded wait on an mbarrier phase (try_wait rounds, each suspending for at most ~1 us);
// gives up at once when another thread of the CTA already gave up.
__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity, int *fail) {
  for (uint32_t it = 0; it < kWaitRounds; ++it) {
    if (*(volatile int *)fail) return false;
    if (umma::mbar_try_wait_hint(bar, parity, 1000)) return true;
  }
  *(volatile int *)fail = 1;
  return false;
}

template <class TX, bool GRAM>
__global__ void __launch_bounds__(kTR, TcCfg<GRAM>::CTAS) trsm_tc_kernel(TcTrsmArgs a) {
  using C = TcCfg<GRAM>;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *Qs = smem;                                           // slice buffer, K-major core matrices
  unsigned char *Rs = smem + C::OFF_R;                                // 3 slices of R (B operands)
  float *Rd = reinterpret_cast<float *>(smem + C::OFF_RD);            // diagonal blocks, Rd[J][c][i]
  float *Ds = reinterpret_cast<float *>(smem + C::OFF_DS);            // fl32(1 / R_jj)
  float *Sc = Ds + 64, *Isc = Sc + 64;                                // Gram split scales per column
  unsigned *Wmax = reinterpret_cast<unsigned *>(smem + C::OFF_WMAX);  // per-warp column maxima (4 x 64)
  int *Src = reinterpret_cast<int *>(smem + C::OFF_SRC);              // source column of X per column
  __shared__ uint64_t bar_upd, bar_gram, bar_drain;
  __shared__ uint32_t tslot;
  __shared__ int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const TX *X = static_cast<const TX *>(a.X);
  const int r = a.rank ? (int)(*a.rank < (int64_t)a.n ? *a.rank : (int64_t)a.n) : a.n;

  // ---- set-up: R pieces (column j, row i at byte (j/8) SBO + (i/8) 128 + (j%8) 16 + (i%8) 2)
  for (int e = tid; e < kTN * kTN / 2; e += kTR) {
    const int j = e / (kTN / 2), i = 2 * (e % (kTN / 2));
    uint32_t h, mm, l;
    split3(a.Rf[i + j * kTN], a.Rf[i + 1 + j * kTN], h, mm, l);
    const uint32_t off = (j / 8) * kRSBO + (i / 8) * 128 + (j % 8) * 16 + (i % 8) * 2;
    *reinterpret_cast<uint32_t *>(Rs + off) = h;
    *reinterpret_cast<uint32_t *>(Rs + kRSlice + off) = mm;
    *reinterpret_cast<uint32_t *>(Rs + 2 * kRSlice + off) = l;
  }
  for (int e = tid; e < 4 * 256; e += kTR) {
    const int J = e >> 8, c = (e >> 4) & 15, i = e & 15;
    Rd[e] = a.Rf[(16 * J + i) + (16 * J + c) * kTN];
  }
  for (int j = tid; j < kTN; j += kTR) {
    Ds[j] = a.dinv[j];
    Src[j] = j < r ? (a.perm ? a.perm[j] : j) : -1;
  }
  if (tid == 0) {
    umma::mbar_init(&bar_upd, 1);
    umma::mbar_init(&bar_gram, 1);
    umma::mbar_init(&bar_drain, 1);
    s_fail = 0;
  }
  if (warp == 0) umma::tmem_alloc(&tslot, C::NCOLS);
  umma::fence_proxy_async();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tbase = tslot;
  const uint32_t lane_base = tbase + ((uint32_t)(32 * warp) << 16);
  const uint32_t qs_addr = umma::smem_u32(Qs), rs_addr = umma::smem_u32(Rs);
  const int n = a.n;

  float accS[GRAM ? 64 : 1], cmpS[GRAM ? 64 : 1];
#pragma unroll
  for (int j = 0; j < (GRAM ? 64 : 1); ++j) accS[j] = cmpS[j] = 0.0f;

  uint32_t ph_upd = 0, ph_gram = 0;
  bool gram_pending = false;
  const int64_t tiles = (a.m + kTR - 1) / kTR;
  const uint32_t row_sw = (uint32_t)(tid / 8) * C::QSBO + (uint32_t)(tid % 8) * 16;   // this row's core offset

  // folds the finished Gram MMAs of the previous tile (TMEM P region) into the Kahan sums
  auto fold = [&]() {
    wait_bar(&bar_gram, ph_gram, &s_fail);   // on a timeout the sums are discarded below
    ph_gram ^= 1u;
    umma::fence_after_sync();
#pragma unroll
    for (int c16 = 0; c16 < 4; ++c16) {
      uint32_t v0[16], v1[16];
      umma::tmem_ld16(lane_base + C::P_COL + 16 * c16, v0);
      umma::tmem_ld16(lane_base + C::P_COL + 64 + 16 * c16, v1);
      umma::tmem_wait_ld();
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int j = 16 * c16 + u;
        const float t = __uint_as_float(v0[u]) + __uint_as_float(v1[u]);
        const float y = t - cmpS[j];
        const float s = accS[j] + y;
        cmpS[j] = (s - accS[j]) - y;
        accS[j] = s;
      }
    }
  };

  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t row = tile * kTR + tid;
    const bool live = row < a.m;
    if constexpr (GRAM) {
      // the previous tile's Gram (its MMAs also read the slice buffer rewritten below)
      if (gram_pending) fold();
      gram_pending = false;
    }
    float q[kTN];
#pragma unroll
    for (int j = 0; j < kTN; ++j) {
      const int src = Src[j];
      q[j] = (live && src >= 0) ? to_f32v(X[row + (int64_t)src * a.ldx]) : 0.0f;
    }
#pragma unroll
    for (int J = 0; J < 4; ++J) {
      if (J > 0) {
        // y_J = x_J - (the tensor-core sum of the earlier blocks' products)
        wait_bar(&bar_upd, ph_upd, &s_fail);
        ph_upd ^= 1u;
        umma::fence_after_sync();
        uint32_t v[16];
        umma::tmem_ld16(lane_base + 16 * (J - 1), v);
        umma::tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 16; ++c) q[16 * J + c] -= __uint_as_float(v[c]);
      }
      // substitution against the diagonal block R_{J,J}: column c of the block is 16 floats
      // at rd + 16 c (read as float4), each dot product in two interleaved FMA chains
      const float4 *rd4 = reinterpret_cast<const float4 *>(Rd + 256 * J);
      const float4 *ds4 = reinterpret_cast<const float4 *>(Ds + 16 * J);
      float dj[16];
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) {
        const float4 d = ds4[c4];
        dj[4 * c4] = d.x; dj[4 * c4 + 1] = d.y; dj[4 * c4 + 2] = d.z; dj[4 * c4 + 3] = d.w;
      }
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        float s0 = q[16 * J + c], s1 = 0.0f;
#pragma unroll
        for (int i4 = 0; i4 < (c + 3) / 4; ++i4) {
          const float4 rv = rd4[4 * c + i4];
          const float rr[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = 4 * i4 + u;
            if (i < c) {
              if (u & 1) s1 = fmaf(-q[16 * J + i], rr[u], s1);
              else s0 = fmaf(-q[16 * J + i], rr[u], s0);
            }
          }
        }
        q[16 * J + c] = (s0 + s1) * dj[c];
      }
      if (J < 3) {
        // the exact three-way split of q_J into the slice buffer (two 16-byte chunks per piece)
#pragma unroll
        for (int h8 = 0; h8 < 2; ++h8) {
          uint32_t hw[4], mw[4], lw[4];
#pragma unroll
          for (int p = 0; p < 4; ++p) split3(q[16 * J + 8 * h8 + 2 * p], q[16 * J + 8 * h8 + 2 * p + 1], hw[p], mw[p], lw[p]);
          const uint32_t col = 16 * J + 8 * h8;
          *reinterpret_cast<uint4 *>(Qs + row_sw + ((0 * C::CW + col) / 8) * 128) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          *reinterpret_cast<uint4 *>(Qs + row_sw + ((1 * C::CW + col) / 8) * 128) = make_uint4(mw[0], mw[1], mw[2], mw[3]);
          *reinterpret_cast<uint4 *>(Qs + row_sw + ((2 * C::CW + col) / 8) * 128) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        umma::fence_proxy_async();
        umma::fence_before_sync();
        __syncthreads();
        if (tid == 0 && !*(volatile int *)&s_fail) {
          umma::fence_after_sync();
          const int N = 16 * (3 - J);
          const uint32_t id = umma::idesc_bf16_f32(128, N);
          // (q piece, R piece) pairs with index sum <= 2
          const int pa[6] = {0, 0, 1, 0, 1, 2}, pr[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
          for (int p = 0; p < 6; ++p) {
            const uint64_t ad = umma::smem_desc(qs_addr + ((pa[p] * C::CW + 16 * J) / 8) * 128, 128, C::QSBO);
            const uint64_t bd = umma::smem_desc(rs_addr + pr[p] * kRSlice + (16 * (J + 1) / 8) * kRSBO + (16 * J / 8) * 128,
                                                128, kRSBO);
            umma::mma_bf16(tbase + 16 * J, ad, bd, id, (J == 0 && p == 0) ? 0u : 1u);
          }
          umma::mma_commit(&bar_upd);
        }
      }
    }
    // the row of Q (columns < n)
    if (live) {
      int64_t ldq = a.ldq;
      asm volatile("" : "+l"(ldq));
#pragma unroll
      for (int j = 0; j < kTN; ++j)
        if (j < n) a.Q[row + (int64_t)j * ldq] = q[j];
    }
    if constexpr (GRAM) {
      // per column, the tile's largest |q| (magnitude bits order like the values)
#pragma unroll
      for (int j = 0; j < kTN; ++j) {
        const unsigned mx = __reduce_max_sync(0xffffffffu, __float_as_uint(q[j]) & 0x7FFFFFFFu);
        if (lane == 0) Wmax[warp * 64 + j] = mx;
      }
      __syncthreads();
      if (tid < kTN) {
        const unsigned mx = max(max(Wmax[tid], Wmax[64 + tid]), max(Wmax[128 + tid], Wmax[192 + tid]));
        const int be = (int)(mx >> 23);           // biased exponent of the largest |q|
        // 2^(6 - e) and 2^(e - 6), e = be - 127; tiny or zero columns keep h = 0 (all in m, l)
        const bool ok = be >= 40 && be <= 200;
        Sc[tid] = ok ? __uint_as_float((uint32_t)(127 + 133 - be) << 23) : 0.0f;
        Isc[tid] = ok ? __uint_as_float((uint32_t)(be - 6) << 23) : 0.0f;
      }
      __syncthreads();
#pragma unroll
      for (int c8 = 0; c8 < kTN / 8; ++c8) {
        uint32_t hw[4], mw[4], lw[4];
        const float4 sa = reinterpret_cast<const float4 *>(Sc)[2 * c8], sb = reinterpret_cast<const float4 *>(Sc)[2 * c8 + 1];
        const float4 ia = reinterpret_cast<const float4 *>(Isc)[2 * c8], ib = reinterpret_cast<const float4 *>(Isc)[2 * c8 + 1];
        const float sc8[8] = {sa.x, sa.y, sa.z, sa.w, sb.x, sb.y, sb.z, sb.w};
        const float is8[8] = {ia.x, ia.y, ia.z, ia.w, ib.x, ib.y, ib.z, ib.w};
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const int j = 8 * c8 + 2 * p;
          split_fixed(q[j], q[j + 1], sc8[2 * p], sc8[2 * p + 1], is8[2 * p], is8[2 * p + 1], hw[p], mw[p], lw[p]);
        }
        const uint32_t col = 8 * c8;
        *reinterpret_cast<uint4 *>(Qs + row_sw + ((0 * C::CW + col) / 8) * 128) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4 *>(Qs + row_sw + ((1 * C::CW + col) / 8) * 128) = make_uint4(mw[0], mw[1], mw[2], mw[3]);
        *reinterpret_cast<uint4 *>(Qs + row_sw + ((2 * C::CW + col) / 8) * 128) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      }
      umma::fence_proxy_async();
      umma::fence_before_sync();
      __syncthreads();
      if (tid == 0 && !*(volatile int *)&s_fail) {
        umma::fence_after_sync();
        const uint32_t idP = idesc_bf16_f32_mn(128, 128), idL = idesc_bf16_f32_mn(128, 64);
        const bool first = tile == blockIdx.x;
#pragma unroll
        for (int t = 0; t < kTR / 16; ++t) {
          // MN-major views: 8-column groups 128 B apart (SBO), 8-row groups QSBO apart (LBO)
          const uint32_t kofs = (uint32_t)(2 * t) * C::QSBO;
          const uint64_t ad = umma::smem_desc(qs_addr + kofs, C::QSBO, 128);           // [h; m]^T
          const uint64_t bl = umma::smem_desc(qs_addr + kofs + (2 * C::CW / 8) * 128, C::QSBO, 128);   // l
          umma::mma_bf16(tbase + C::P_COL, ad, ad, idP, t > 0 ? 1u : 0u);
          umma::mma_bf16(tbase + C::L_COL, ad, bl, idL, (t > 0 || !first) ? 1u : 0u);
        }
        umma::mma_commit(&bar_gram);
      }
      gram_pending = true;
    }
  }

  if constexpr (GRAM) {
    if (gram_pending) fold();
    // per-CTA partial: G = S + T + Lh + Lm + Lh^T + Lm^T (rows of S, Lh in lanes 0..63;
    // of T, Lm in lanes 64..127), assembled in FP64 in shared memory (the slice buffer and
    // the R pieces are free now), in phases so that no two threads add to one entry at once
    umma::fence_after_sync();
    double *F = reinterpret_cast<double *>(Qs);     // 64 x 64, F[i * 64 + j]
    const int i = tid & 63;
    __syncthreads();
    if (tid < 64) {
#pragma unroll
      for (int j = 0; j < 64; ++j) F[i * 64 + j] = (double)accS[j] - (double)cmpS[j];
    }
    __syncthreads();
    if (tid >= 64) {
#pragma unroll
      for (int j = 0; j < 64; ++j) F[i * 64 + j] += (double)accS[j] - (double)cmpS[j];
    }
    // the small terms, 16 TMEM columns at a time: rows (Lh, Lm), then columns (Lh^T, Lm^T)
#pragma unroll 1
    for (int ph = 0; ph < 4; ++ph) {
      __syncthreads();
      const bool mine = (ph & 1) ? tid >= 64 : tid < 64;
      if (mine) {
#pragma unroll
        for (int c16 = 0; c16 < 4; ++c16) {
          uint32_t v[16];
          umma::tmem_ld16(lane_base + C::L_COL + 16 * c16, v);
          umma::tmem_wait_ld();
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int j = 16 * c16 + u;
            if (ph < 2) F[i * 64 + j] += (double)__uint_as_float(v[u]);
            else F[j * 64 + i] += (double)__uint_as_float(v[u]);
          }
        }
      }
    }
    __syncthreads();
    double *pb = a.partial + (int64_t)blockIdx.x * n * n;
    const double nan = __longlong_as_double(0x7FF8000000000000ll);
    const bool failed = *(volatile int *)&s_fail != 0;
    for (int e = tid; e < n * n; e += kTR) {
      const int ii = e % n, jj = e / n;
      pb[e] = failed ? nan : ((ii <= jj) ? F[ii * 64 + jj] : 0.0);
    }
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

template <bool GRAM>
int tc_grid(int64_t m) {
  const int64_t tiles = (m + kTR - 1) / kTR;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)TcCfg<GRAM>::CTAS * num_sms()));
}

template <class TX, bool GRAM>
cudaError_t launch_tc(const TcTrsmArgs &a, int grid, cudaStream_t st) {
  auto kern = trsm_tc_kernel<TX, GRAM>;
  cudaError_t e = set_smem(kern, TcCfg<GRAM>::SMEM);
  if (e != cudaSuccess) return e;
  kern<<<grid, kTR, TcCfg<GRAM>::SMEM, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

bool trsm_tc_supported(int64_t n) { return n > 32 && n <= 64; }

int trsm_tc_gram_groups(int64_t m) { return tc_grid<true>(m); }

cudaError_t launch_trsm_tc_gram(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, const float *Rf,
                                const float *dinv, const int32_t *perm, const int64_t *rank, float *Q, int64_t ldq,
                                double *partial, int *status, cudaStream_t st) {
  TcTrsmArgs a{X, m, (int)n, ldx, Rf, dinv, perm, rank, Q, ldq, partial, status};
  const int grid = tc_grid<true>(m);
  return prec == RCQR_BF16 ? launch_tc<__nv_bfloat16, true>(a, grid, st) : launch_tc<float, true>(a, grid, st);
}

}  // namespace rcqr
