// Sketch P = Theta X (Alg. 2 step 1) on the tcgen05 tensor cores, exact.
//
// Theta's entries are the integer levels T[t] in [-127, 127] (scaled by
// 1/sqrt(k v) afterwards), i.e. 7-bit integers, exact in bf16.  X is cut, per
// 1024-row block and column, into S signed 7-bit integer slices relative to
// the block's largest exponent e (x = sum_b s_b 2^(e-6-7b) + a remainder below
// the last slice; an error-free splitting in the manner of Ozaki et al.).
// Each slice is a bf16 operand; every product T*s is an integer below 2^14,
// so the fp32 tensor-core sums over at most 1024 rows stay below 2^24 and
// are exact.  The first NE slices get their own TMEM accumulators (exact);
// the remaining ones, pre-scaled by 2^-7 per slice, share one accumulator
// whose fp32 rounding over a block stays ~2^-39 (FP32 X: 3 exact of 5
// slices) / 2^-46 (FP64 X: 4 exact of 8) below the block's largest |x|;
// BF16 X needs 3 slices and its last one alone is exact as well.
// After every block the accumulators are read from TMEM, combined into one
// int64 per entry and added into a per-column block-floating-point int64
// accumulator in registers (the "simple addition" of Sec. 3.1 done exactly,
// up to one truncation of ~2^-52 relative per block).
//
// Per CTA: a contiguous run of blocks (split-K over m), KCH chunks of 128
// rows of Theta and NC columns of X.  Per stage of BK rows: all 512 threads
// generate the Theta tile (Philox4x32-10 + level table) and the X slices in
// shared memory in the K-major core-matrix layout; one thread issues the
// MMAs (M = 128, N = NC, K = 16) and commits them to the stage's mbarrier;
// two stages let the tensor core work on one while the CUDA cores fill the
// other.  Every wait is bounded; a timeout marks the partial sums NaN and
// raises RCQR_ETIMEOUT in the status word.
#include <algorithm>

#include "common.cuh"
#include "rcqr_internal.h"
#include "theta.cuh"
#include "umma.cuh"

namespace rcqr {

__constant__ int8_t c_theta_levels[256];

namespace {

constexpr int kThreadsTC = 512;
constexpr int kBlockRows = 1024;      // rows per exponent block / TMEM promotion
constexpr int kStages = 2;
constexpr uint32_t kWaitPolls = 1u << 26;

template <int PREC>
struct SliceCfg;
// S slices; the first NE have exact accumulators, the rest share one (weights
// 2^-7 apart); LS fractional bits of that shared accumulator are kept in the
// int64 sum.  Headroom: 24 + 7 NE + LS + log2(MAXB) <= 62 bits.
template <>
struct SliceCfg<RCQR_F64> {
  using T = double;
  static constexpr int S = 8, NE = 4, LS = 4, MAXB = 64;
};
template <>
struct SliceCfg<RCQR_F32> {
  using T = float;
  static constexpr int S = 5, NE = 3, LS = 10, MAXB = 128;
};
template <>
struct SliceCfg<RCQR_BF16> {
  using T = __nv_bfloat16;
  static constexpr int S = 3, NE = 2, LS = 8, MAXB = 128;
};

struct TcArgs {
  const void *X;
  int64_t m;
  int n;
  int64_t ldx;
  int k;
  uint64_t seed;
  uint32_t stream_id;
  int64_t row_offset;
  int64_t blk0;    // first 1024-row block (global index)
  int64_t nblk;    // blocks covering [row_offset, row_offset + m)
  int groups;      // CTAs along m
  int NC;          // columns per CTA (multiple of 16)
  int ngrp;        // column groups
  int KCH;         // 128-row chunks of Theta per CTA
  int BK;          // rows per stage (16, 32 or 64)
  double *partial; // [groups][n][k]
  int *status;     // nullable
};

constexpr int EMPTY_EXP = -0x40000000;

__device__ __forceinline__ uint32_t abs_bits(float x) { return __float_as_uint(x) & 0x7FFFFFFFu; }

// Exponent of the largest |x| of a block column: returns EMPTY_EXP for an all-zero column.
__device__ __forceinline__ int block_exp_f32(uint32_t maxbits) {
  const int be = (int)(maxbits >> 23);
  return be == 0 ? EMPTY_EXP : be - 127;     // zero or subnormal-only column: treated as zero
}
__device__ __forceinline__ int block_exp_f64(unsigned long long maxbits) {
  const int be = (int)((maxbits >> 52) & 0x7FF);
  return be == 0 ? EMPTY_EXP : be - 1023;
}

__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(e + 127) << 23); }

// Writes the S slices of 8 consecutive rows of one column (bf16, 16 bytes per
// slice) to dst + b * slice_stride.  e is the block's column exponent.
template <int PREC>
__device__ __forceinline__ void slice8_store(const typename SliceCfg<PREC>::T (&x)[8], int e, unsigned char *dst,
                                             int slice_stride) {
  constexpr int S = SliceCfg<PREC>::S, NE = SliceCfg<PREC>::NE;
  if constexpr (PREC == RCQR_F64) {
    unsigned long long F[8];
    uint32_t neg = 0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const unsigned long long bits = (unsigned long long)__double_as_longlong(x[t]);
      const int be = (int)((bits >> 52) & 0x7FF);
      neg |= (uint32_t)(bits >> 63) << t;
      unsigned long long f = 0;
      if (be != 0 && e != EMPTY_EXP) {
        const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int d = e - (be - 1023);           // >= 0: x is not larger than the block maximum
        f = d <= 3 ? (mant << (3 - d)) : (d - 3 < 64 ? (mant >> (d - 3)) : 0ull);
      }
      F[t] = f;                                  // |x| * 2^(55-e), below 2^56
    }
#pragma unroll
    for (int b = 0; b < S; ++b) {
      uint32_t w[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        uint32_t h[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int t = 2 * p + q;
          const uint32_t dig = (uint32_t)(F[t] >> (49 - 7 * b)) & 127u;
          float v = __uint_as_float(0x4B000000u | dig) - 8388608.0f;   // the digit, exactly
          if (b >= NE) v *= pow2f(-7 * (b - NE));
          if ((neg >> t) & 1u) v = -v;
          h[q] = __float_as_uint(v) >> 16;
        }
        w[p] = h[0] | (h[1] << 16);
      }
      *reinterpret_cast<uint4 *>(dst + b * slice_stride) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  } else {
    // FP32 / BF16 storage: scale into (-128, 128) and peel off rounded 7-bit digits
    float t8[8];
    const int sh = 6 - e;
    const float s1 = pow2f(sh / 2), s2 = pow2f(sh - sh / 2);
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      float xv;
      if constexpr (PREC == RCQR_BF16)
        xv = __bfloat162float(x[t]);
      else
        xv = x[t];
      if (e == EMPTY_EXP || abs_bits(xv) < 0x00800000u) xv = 0.0f;
      t8[t] = (xv * s1) * s2;
    }
#pragma unroll
    for (int b = 0; b < S; ++b) {
      uint32_t w[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        uint32_t h[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int t = 2 * p + q;
          const float d = rintf(t8[t]);
          if (b + 1 < S) t8[t] = (t8[t] - d) * 128.0f;
          float v = d;
          if (b >= NE) v *= pow2f(-7 * (b - NE));
          h[q] = __float_as_uint(v) >> 16;
        }
        w[p] = h[0] | (h[1] << 16);
      }
      *reinterpret_cast<uint4 *>(dst + b * slice_stride) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

template <int PREC, int KCH, int JCH>
__global__ void __launch_bounds__(kThreadsTC, 1) sketch_tc_kernel(TcArgs a) {
  using T = typename SliceCfg<PREC>::T;
  constexpr int S = SliceCfg<PREC>::S, NE = SliceCfg<PREC>::NE, LS = SliceCfg<PREC>::LS;
  constexpr int NACC = NE + 1;
  constexpr int NC = 64 * JCH;                 // columns per CTA
  constexpr int CW = 16 * JCH;                 // columns per thread in the promotion
  constexpr uint32_t NCOLS = (KCH * NACC * NC) <= 256 ? 256u : 512u;
  static_assert(KCH * NACC * NC <= 512, "TMEM holds 512 columns");
  static_assert(24 + 7 * NE + LS + 7 <= 62 || SliceCfg<PREC>::MAXB <= 64, "int64 headroom");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t bars[kStages];
  __shared__ uint32_t tslot;
  __shared__ int e_col[NC];        // this block's column exponents
  __shared__ int E_col[NC];        // running exponents of the int64 accumulators
  __shared__ int s_fail;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int BK = a.BK;
  const int g = blockIdx.y;
  const int kgi = blockIdx.x / a.ngrp, ngi = blockIdx.x % a.ngrp;
  const int col0 = ngi * NC;
  const T *X = static_cast<const T *>(a.X);

  // shared memory: level table replicated per lane (bank = lane), then the stages
  uint32_t *table = reinterpret_cast<uint32_t *>(smem_raw);
  unsigned char *stage_base = smem_raw + 256 * 32 * 4;
  const int a_bytes = KCH * 128 * BK * 2;
  const int b_bytes = S * NC * BK * 2;
  const int stage_bytes = a_bytes + b_bytes;

  for (int e = tid; e < 256 * 32; e += blockDim.x) {
    const int lev = (int)c_theta_levels[e >> 5];
    table[e] = __float_as_uint((float)lev) >> 16;
  }
  for (int j = tid; j < NC; j += blockDim.x) E_col[j] = EMPTY_EXP;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) umma::mbar_init(&bars[s], 1);
    s_fail = 0;
  }
  if (warp == 0) umma::tmem_alloc(&tslot, NCOLS);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tbase = tslot;

  // this thread's accumulators: TMEM lane 32*(warp%4)+lane (a row of Theta within
  // each chunk) and columns [cq*CW, cq*CW+CW)
  const int lq = warp & 3, cq = warp >> 2;
  long long A[KCH][CW];
#pragma unroll
  for (int c = 0; c < KCH; ++c)
#pragma unroll
    for (int j = 0; j < CW; ++j) A[c][j] = 0;

  const int64_t bb = a.blk0 + (a.nblk * g) / a.groups;
  const int64_t be_ = a.blk0 + (a.nblk * (g + 1)) / a.groups;
  const uint32_t idesc = umma::idesc_bf16_f32(128, NC);
  const int steps_per_block = kBlockRows / BK;
  int it = 0;

  for (int64_t blk = bb; blk < be_; ++blk) {
    const int64_t grow0 = blk * kBlockRows;
    // ---- exponent pass: the largest |x| of each column over the block
    for (int jl = warp; jl < NC; jl += kThreadsTC / 32) {
      const int j = col0 + jl;
      if constexpr (PREC == RCQR_F64) {
        unsigned long long mx = 0;
        if (j < a.n)
          for (int r = lane; r < kBlockRows; r += 32) {
            const int64_t lr = grow0 + r - a.row_offset;
            if (lr >= 0 && lr < a.m) {
              const unsigned long long bits = (unsigned long long)__double_as_longlong(X[lr + (int64_t)j * a.ldx]);
              mx = max(mx, bits & 0x7FFFFFFFFFFFFFFFull);
            }
          }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) e_col[jl] = block_exp_f64(mx);
      } else {
        uint32_t mx = 0;
        if (j < a.n)
          for (int r = lane; r < kBlockRows; r += 32) {
            const int64_t lr = grow0 + r - a.row_offset;
            if (lr >= 0 && lr < a.m) {
              float v;
              if constexpr (PREC == RCQR_BF16)
                v = __bfloat162float(X[lr + (int64_t)j * a.ldx]);
              else
                v = X[lr + (int64_t)j * a.ldx];
              mx = max(mx, abs_bits(v));
            }
          }
        mx = __reduce_max_sync(0xffffffffu, mx);
        if (lane == 0) e_col[jl] = block_exp_f32(mx);
      }
    }
    __syncthreads();

    for (int st = 0; st < steps_per_block; ++st, ++it) {
      const int sidx = it % kStages;
      unsigned char *sA = stage_base + sidx * stage_bytes;
      unsigned char *sB = sA + a_bytes;
      if (it >= kStages) {
        if (!umma::mbar_wait(&bars[sidx], (uint32_t)((it / kStages - 1) & 1), kWaitPolls)) s_fail = 1;
      }
      const int64_t r0 = grow0 + (int64_t)st * BK;
      // ---- Theta tile: KCH*128 rows x BK columns, 16 columns per Philox call
      const int cpr = BK / 16;
      for (int cidx = tid; cidx < KCH * 128 * cpr; cidx += kThreadsTC) {
        const int qq = cidx % cpr;
        const int row = cidx / cpr;
        const int c = row >> 7, il = row & 127;
        const int i = (kgi * KCH + c) * 128 + il;
        uint32_t wv[8];
        if (i < a.k) {
          const uint4 w = theta_block((uint64_t)(r0 / 16 + qq), (uint32_t)i, a.stream_id, a.seed);
          const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            const uint32_t b0 = (ww[p >> 1] >> (16 * (p & 1))) & 0xFFu;
            const uint32_t b1 = (ww[p >> 1] >> (16 * (p & 1) + 8)) & 0xFFu;
            wv[p] = table[b0 * 32 + lane] | (table[b1 * 32 + lane] << 16);
          }
        } else {
#pragma unroll
          for (int p = 0; p < 8; ++p) wv[p] = 0u;
        }
        unsigned char *dst = sA + c * (128 * BK * 2) + (il >> 3) * (BK * 16) + (il & 7) * 16;
        *reinterpret_cast<uint4 *>(dst + (2 * qq) * 128) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        *reinterpret_cast<uint4 *>(dst + (2 * qq + 1) * 128) = make_uint4(wv[4], wv[5], wv[6], wv[7]);
      }
      // ---- X slices: S operands of NC x BK; one thread per 8-row octet of a column
      const int opc = BK / 8;
      for (int o = tid; o < NC * opc; o += kThreadsTC) {
        const int oc = o % opc, jl = o / opc;
        const int j = col0 + jl;
        T xv[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int64_t lr = r0 + 8 * oc + t - a.row_offset;
          xv[t] = (j < a.n && lr >= 0 && lr < a.m) ? X[lr + (int64_t)j * a.ldx] : T(0);
        }
        unsigned char *dst = sB + (jl >> 3) * (BK * 16) + oc * 128 + (jl & 7) * 16;
        slice8_store<PREC>(xv, j < a.n ? e_col[jl] : EMPTY_EXP, dst, NC * BK * 2);
      }
      umma::fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        umma::fence_after_sync();
        const uint32_t a0 = umma::smem_u32(sA), b0 = umma::smem_u32(sB);
#pragma unroll
        for (int c = 0; c < KCH; ++c)
#pragma unroll
          for (int b = 0; b < S; ++b) {
            const int acc = b < NE ? b : NE;
            const uint32_t dcol = tbase + (uint32_t)((c * NACC + acc) * NC);
            for (int q = 0; q < BK / 16; ++q) {
              const uint64_t ad = umma::smem_desc(a0 + c * (128 * BK * 2) + q * 256, 128, BK * 16);
              const uint64_t bd = umma::smem_desc(b0 + b * (NC * BK * 2) + q * 256, 128, BK * 16);
              const bool first = (st == 0) && (q == 0) && (b <= NE);
              umma::mma_bf16(dcol, ad, bd, idesc, first ? 0u : 1u);
            }
          }
        umma::mma_commit(&bars[sidx]);
      }
    }
    // ---- promotion: wait for the block's last MMAs, fold TMEM into the int64 accumulators
    {
      const int last = (it - 1) % kStages;
      if (!umma::mbar_wait(&bars[last], (uint32_t)(((it - 1) / kStages) & 1), kWaitPolls)) s_fail = 1;
    }
    umma::fence_after_sync();
#pragma unroll
    for (int jc0 = 0; jc0 < CW; jc0 += 16) {
#pragma unroll
      for (int c = 0; c < KCH; ++c) {
        uint32_t rv[NACC][16];
#pragma unroll
        for (int acc = 0; acc < NACC; ++acc)
          umma::tmem_ld16(tbase + ((uint32_t)(32 * lq) << 16) + (uint32_t)((c * NACC + acc) * NC + cq * CW + jc0),
                          rv[acc]);
        umma::tmem_wait_ld();
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int jl = cq * CW + jc0 + jj;
          const int e = e_col[jl];
          if (e == EMPTY_EXP) continue;
          long long V = 0;
#pragma unroll
          for (int b = 0; b < NE; ++b)
            V += (long long)__float2int_rn(__uint_as_float(rv[b][jj])) << (7 * (NE - b) + LS);
          V += __float2ll_rn(__uint_as_float(rv[NE][jj]) * (float)(1 << LS));
          const int f = e - 6 - 7 * NE - LS;
          const int Ec = E_col[jl];
          long long acc_v = A[c][jc0 + jj];
          if (Ec == EMPTY_EXP) {
            acc_v = V;
          } else if (f >= Ec) {
            const int sh = f - Ec;
            acc_v = (sh >= 63 ? (acc_v < 0 ? -1LL : 0LL) : (acc_v >> sh)) + V;
          } else {
            const int sh = Ec - f;
            acc_v += sh >= 63 ? (V < 0 ? -1LL : 0LL) : (V >> sh);
          }
          A[c][jc0 + jj] = acc_v;
        }
      }
    }
    umma::fence_before_sync();
    __syncthreads();
    // running exponent of each column: the larger of the old one and this block's frame
    for (int jl = tid; jl < NC; jl += blockDim.x) {
      const int e = e_col[jl];
      if (e == EMPTY_EXP) continue;
      const int f = e - 6 - 7 * NE - LS;
      if (E_col[jl] == EMPTY_EXP || f > E_col[jl]) E_col[jl] = f;
    }
    __syncthreads();
  }

  // ---- this CTA's partial sketch: partial[g][j][i]
  const bool failed = s_fail != 0;
#pragma unroll
  for (int c = 0; c < KCH; ++c) {
    const int i = (kgi * KCH + c) * 128 + lq * 32 + lane;
#pragma unroll
    for (int jc = 0; jc < CW; ++jc) {
      const int jl = cq * CW + jc;
      const int j = col0 + jl;
      if (i >= a.k || j >= a.n) continue;
      const int Ec = E_col[jl];
      double v = Ec == EMPTY_EXP ? 0.0 : ldexp((double)A[c][jc], Ec);
      if (failed) v = __longlong_as_double(0x7FF8000000000000ll);
      a.partial[((int64_t)g * a.n + j) * a.k + i] = v;
    }
  }
  if (failed && tid == 0 && a.status) {
    a.status[0] = RCQR_ETIMEOUT;
    a.status[1] = -1;
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tbase, NCOLS);
}

// P(i, j) = c * sum_g partial[g](i, j): one warp per entry, fixed order.
__global__ void sketch_tc_reduce_kernel(const double *__restrict__ partial, int groups, int k, int n,
                                        double c, double *__restrict__ P, int64_t ldp) {
  const int64_t idx = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (idx >= (int64_t)k * n) return;
  const int i = (int)(idx % k), j = (int)(idx / k);
  const double s = warp_sum_strided(partial + (int64_t)j * k + i, groups, (int64_t)n * k);
  if ((threadIdx.x & 31) == 0) P[i + (int64_t)j * ldp] = c * s;
}

struct TcPlan {
  int JCH, NC, ngrp, KCH, kgrp, BK, groups, S;
  int64_t blk0, nblk;
  size_t smem;
};

TcPlan plan_tc(int64_t m, int64_t n, int64_t k, int64_t row_offset, int prec) {
  TcPlan p{};
  p.S = prec == RCQR_F64 ? 8 : (prec == RCQR_F32 ? 5 : 3);
  const int nacc = prec == RCQR_F64 ? 5 : (prec == RCQR_F32 ? 4 : 3);
  const int maxb = prec == RCQR_F64 ? 64 : 128;
  // columns per CTA: 64 or 128; TMEM (512 columns) holds nacc accumulators of
  // NC columns for each of the KCH chunks of 128 Theta rows
  const int ncmax = nacc * 128 <= 512 ? 128 : 64;
  p.ngrp = (int)((n + ncmax - 1) / ncmax);
  const int64_t per_group = (n + p.ngrp - 1) / p.ngrp;
  p.JCH = per_group > 64 ? 2 : 1;
  p.NC = 64 * p.JCH;
  const int kchunks = (int)((k + 127) / 128);
  p.KCH = (p.JCH == 1 && kchunks >= 2 && 2 * nacc * 64 <= 512) ? 2 : 1;
  p.kgrp = (kchunks + p.KCH - 1) / p.KCH;
  // rows per stage: the largest of 64/32/16 whose two stages fit beside the table
  const size_t table = 256 * 32 * 4;
  p.BK = 64;
  auto bytes = [&](int bk) {
    return table + (size_t)kStages * ((size_t)p.KCH * 128 * bk * 2 + (size_t)p.S * p.NC * bk * 2);
  };
  while (p.BK > 16 && bytes(p.BK) > 200 * 1024) p.BK /= 2;
  p.smem = bytes(p.BK);
  p.blk0 = row_offset / kBlockRows;
  p.nblk = (row_offset + m + kBlockRows - 1) / kBlockRows - p.blk0;
  const int64_t ctas_per_rows = (int64_t)p.kgrp * p.ngrp;
  int64_t groups = std::max<int64_t>(1, num_sms() / ctas_per_rows);
  groups = std::min<int64_t>(groups, p.nblk);
  groups = std::max<int64_t>(groups, (p.nblk + maxb - 1) / maxb);
  p.groups = (int)std::min<int64_t>(groups, 65535);
  return p;
}

template <int PREC, int KCH, int JCH>
cudaError_t launch_tc_variant(const TcArgs &a, dim3 grid, size_t smem, cudaStream_t st) {
  auto kern = sketch_tc_kernel<PREC, KCH, JCH>;
  cudaError_t e = set_smem(kern, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreadsTC, smem, st>>>(a);
  return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_tc_prec(const TcArgs &a, const TcPlan &p, dim3 grid, cudaStream_t st) {
  if constexpr (PREC == RCQR_F64) {
    return launch_tc_variant<PREC, 1, 1>(a, grid, p.smem, st);
  } else {
    if (p.JCH == 2) return launch_tc_variant<PREC, 1, 2>(a, grid, p.smem, st);
    if (p.KCH == 2) return launch_tc_variant<PREC, 2, 1>(a, grid, p.smem, st);
    return launch_tc_variant<PREC, 1, 1>(a, grid, p.smem, st);
  }
}

}  // namespace

bool sketch_tc_supported(int64_t n, int64_t k) {
  (void)k;
  return n >= 1 && n <= 256;
}

size_t sketch_tc_workspace(int64_t m, int64_t n, int64_t k, int64_t row_offset, int prec) {
  const TcPlan p = plan_tc(m, n, k, row_offset, prec);
  Workspace w(nullptr, 0);
  w.take<double>((size_t)p.groups * n * k);
  return w.used;
}

cudaError_t launch_sketch_tc(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, int64_t k,
                             uint64_t seed, uint32_t stream_id, int64_t row_offset, double *P,
                             int64_t ldp, int *dev_status, Workspace &ws, cudaStream_t st) {
  static bool table_ready[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !table_ready[dev]) {
    cudaError_t e = cudaMemcpyToSymbol(c_theta_levels, theta_table().level, 256);
    if (e != cudaSuccess) return e;
    table_ready[dev] = true;
  }
  const TcPlan p = plan_tc(m, n, k, row_offset, prec);
  double *partial = ws.take<double>((size_t)p.groups * n * k);
  if (!partial) return cudaErrorMemoryAllocation;
  TcArgs a;
  a.X = X;
  a.m = m;
  a.n = (int)n;
  a.ldx = ldx;
  a.k = (int)k;
  a.seed = seed;
  a.stream_id = stream_id;
  a.row_offset = row_offset;
  a.blk0 = p.blk0;
  a.nblk = p.nblk;
  a.groups = p.groups;
  a.NC = p.NC;
  a.ngrp = p.ngrp;
  a.KCH = p.KCH;
  a.BK = p.BK;
  a.partial = partial;
  a.status = dev_status;
  dim3 grid((unsigned)(p.kgrp * p.ngrp), (unsigned)p.groups);
  cudaError_t e;
  switch (prec) {
    case RCQR_F64: e = launch_tc_prec<RCQR_F64>(a, p, grid, st); break;
    case RCQR_F32: e = launch_tc_prec<RCQR_F32>(a, p, grid, st); break;
    default: e = launch_tc_prec<RCQR_BF16>(a, p, grid, st);
  }
  if (e != cudaSuccess) return e;
  sketch_tc_reduce_kernel<<<(unsigned)((k * n * 32 + 255) / 256), 256, 0, st>>>(partial, p.groups, (int)k, (int)n,
                                                                          theta_scale(k), P, ldp);
  return cudaGetLastError();
}

}  // namespace rcqr
