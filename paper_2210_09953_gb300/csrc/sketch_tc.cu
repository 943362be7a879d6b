// Sketch P = Theta X (Alg. 2 step 1) on the tcgen05 tensor cores, exact.
//
// Theta's entries are the integer levels T[t] in [-127, 127] (scaled by
// 1/sqrt(k v) afterwards), i.e. 7-bit integers, exact in bf16.  X is cut, per
// block of rows and column, into S signed digit slices relative to the
// block's largest exponent e (an error-free splitting in the manner of Ozaki
// et al.):
//   * FP32 / BF16 X: t = x 2^(5-e) in (-64, 64); slice b < S-1 is the
//     remainder rounded to a multiple of 2^(-7b), so every such digit is at most
//     64 units of its slice and every product T d is below 2^13 units: the fp32
//     tensor-core sums over a 2048-row block are exact; the last slice is the
//     remainder rounded to bf16 (it goes to the shared, rounded accumulator);
//   * FP64 X: the truncated 7-bit digits of |x| 2^(55-e), products below 2^14,
//     1024-row blocks.
// Each slice is a bf16 operand with at most 8 significant bits.  The first NE
// slices get their own TMEM accumulators (exact); the remaining ones share one
// accumulator whose fp32 rounding over a block stays ~2^-38 (FP32 X: 3 exact
// of 5 slices) / 2^-46 (FP64 X: 4 exact of 8) below the block's largest |x|;
// BF16 X needs 3 slices.  After every block the accumulators are read from
// TMEM, combined into one int64 per entry and added into a per-column
// block-floating-point int64 accumulator whose exponent is fixed per CTA (the
// largest block exponent of its rows; the "simple addition" of Sec. 3.1 done
// exactly, up to one truncation of ~2^-52 of that column's largest entry per block).
//
// Per CTA: a contiguous run of blocks (split-K over m), KCH chunks of 128
// rows of Theta and NC columns of X.  The CTA's 16 warps are specialised
// around a ring of D shared-memory stages of 32 rows each:
//   * 4 KCH Theta warps generate the Theta tile of a stage (Philox4x32-10 with
//     the round keys as kernel parameters, the level table replicated per lane)
//     in the K-major core-matrix layout;
//   * the other producer warps (12 in all) copy the X rows of a stage three
//     stages ahead into a small ring (cp.async, no registers held), then cut
//     them into slices with the block's column exponents (found beforehand by
//     block_exp_kernel);
//   * warp 15 waits for a stage to be full and issues its MMAs from one thread
//     (M = 128, K = 16; the exact slices of a group stacked along N, up to 256),
//     committing them to the stage's "empty" barrier and, after a block's last
//     stage, to the "accumulators full" barrier;
//   * once a block's MMAs are done, all 16 warps fold TMEM into the int64
//     accumulators (kept in the workspace, L2-resident), four warps per TMEM
//     lane quadrant: warps 12..14 do nothing else, warp 15 after issuing the
//     block's last MMAs, the producers after filling the ring with the next
//     block's first stages (they would wait for a free slot otherwise).
// Every wait is bounded; a timeout marks the partial sums NaN and raises
// RCQR_ETIMEOUT in the status word.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "common.cuh"
#include "rcqr_internal.h"
#include "theta.cuh"
#include "umma.cuh"

namespace rcqr {

namespace {

constexpr int kThreadsTC = 512;                     // 16 warps
constexpr int kProdWarps = 12;                      // warps 0..11 produce (Theta, then X); they arrive on "full";
                                                    // 12..14 only fold; 15 issues the MMAs (all 16 fold)
// Rows per exponent block / TMEM promotion: products T d stay below 2^13
// (FP32/BF16: |d| <= 64) or 2^14 (FP64: 7-bit digits), so the fp32 sums are
// exact over 2048 or 1024 rows.
constexpr int block_rows(int prec) { return prec == RCQR_F64 ? 1024 : 2048; }
constexpr int kBK = 32;                             // rows of X per stage
constexpr int kMaxStages = 6;
constexpr int kTableBytes = 256 * 32 * 4;           // level table, one copy per lane
constexpr uint32_t kWaitPolls = 1u << 22;          // polls with sleeps of up to 256 ns: about 1 s
constexpr int kXAhead = 3;                          // X rows are copied this many stages ahead
constexpr int kXSlots = kXAhead + 1;                // slots of the X copy ring

template <int PREC>
struct SliceCfg;
// S slices; the first NE have exact accumulators, the rest share one; LS
// fractional bits of that shared accumulator are kept in the int64 sum.
// Headroom: 24 + 7 NE + LS + log2(MAXB) <= 62 bits.
template <>
struct SliceCfg<RCQR_F64> {
  using T = double;
  using MaxT = unsigned long long;
  static constexpr int S = 8, NE = 4, LS = 4, MAXB = 64;
};
template <>
struct SliceCfg<RCQR_F32> {
  using T = float;
  using MaxT = uint32_t;
  static constexpr int S = 5, NE = 3, LS = 10, MAXB = 128;
};
template <>
struct SliceCfg<RCQR_BF16> {
  using T = __nv_bfloat16;
  using MaxT = uint32_t;
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
  uint32_t rk[20];    // Philox round keys of the seed (see philox4x32_10_keys)
  int64_t row_offset;
  int64_t blk0;       // first block of rows (global index)
  int64_t nblk;       // blocks covering [row_offset, row_offset + m)
  int groups;         // CTAs along m
  int ngrp;           // column groups
  int D;              // pipeline stages
  int vec;            // X rows may be read 16 bytes at a time
  const int *eblk;    // column exponents of the blocks: eblk[(blk - blk0) * n + j]
  double *partial;    // [groups][n][k]
  long long *acc64;   // int64 accumulators, KCH * NC * 128 per CTA
  int *status;        // nullable
  uint32_t polls;     // bound of every pipeline wait (rounds of poll + sleep)
  ThetaTable theta;   // the 256 levels T[t], passed by value (no device state to set up)
  int dist;           // RCQR_THETA_GAUSSIAN (levels from Philox bytes) or RCQR_THETA_RADEMACHER (bits)
};

constexpr int EMPTY_EXP = -0x40000000;

// Exponent floor(log2 |x|) of the largest |x| of a block column, from its
// magnitude bits (subnormal values included): EMPTY_EXP for an all-zero column.
__device__ __forceinline__ int block_exp(uint32_t maxbits) {
  if (maxbits == 0) return EMPTY_EXP;
  const int be = (int)(maxbits >> 23);
  return be != 0 ? be - 127 : (31 - __clz((int)maxbits)) - 149;
}
__device__ __forceinline__ int block_exp(unsigned long long maxbits) {
  if (maxbits == 0) return EMPTY_EXP;
  const int be = (int)((maxbits >> 52) & 0x7FF);
  return be != 0 ? be - 1023 : (63 - __clzll((long long)maxbits)) - 1074;
}

__device__ __forceinline__ uint32_t mag_bits(float x) { return __float_as_uint(x) & 0x7FFFFFFFu; }
__device__ __forceinline__ uint32_t mag_bits(__nv_bfloat16 x) {
  return ((uint32_t)__bfloat16_as_ushort(x) & 0x7FFFu) << 16;
}
__device__ __forceinline__ unsigned long long mag_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(e + 127) << 23); }

// rint(t) as int64 for an FP32 t with |t| < 2^45, without a 64-bit conversion (those
// run on the FP64 unit, a small fraction of the FP32 rate): t = h 2^24 + l with h the
// nearest integer to t 2^-24 (the 1.5 2^23 addition rounds it; |h| < 2^21) and
// l = t - h 2^24 exact (|l| <= 2^23, a multiple of t's ulp), then rint(l) by one 32-bit
// conversion.  Equal to __float2ll_rn(t): for |t| >= 2^23, t and l are integers; below,
// h = 0 and l = t.
__device__ __forceinline__ long long rint_to_ll(float t) {
  const float hm = fmaf(t, 0x1p-24f, 0x1.8p23f);
  const int h = __float_as_int(hm) - 0x4B400000;
  const float l = fmaf(-(hm - 0x1.8p23f), 0x1p24f, t);
  return ((long long)h << 24) + __float2int_rn(l);
}

// Packed pairs (add.rn.f32x2 / mul.rn.f32x2 of the sm_100 family): two
// independent IEEE round-to-nearest operations in one instruction.
__device__ __forceinline__ void add2(float &d0, float &d1, float a0, float a1, float b0, float b1) {
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d0), "=f"(d1)
      : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}
__device__ __forceinline__ void mul2(float &d0, float &d1, float a0, float a1, float b0, float b1) {
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d0), "=f"(d1)
      : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

// 8 consecutive rows lr0 .. lr0+7 of column j (zeros outside X).
template <class T>
__device__ __forceinline__ void load8(const T *__restrict__ X, int64_t lr0, int j, const TcArgs &a, T (&v)[8]) {
  if (j < a.n && a.vec && lr0 >= 0 && lr0 + 8 <= a.m) {
    const T *p = X + lr0 + (int64_t)j * a.ldx;
    if constexpr (sizeof(T) == 4) {
      const float4 u0 = __ldg(reinterpret_cast<const float4 *>(p));
      const float4 u1 = __ldg(reinterpret_cast<const float4 *>(p) + 1);
      v[0] = u0.x; v[1] = u0.y; v[2] = u0.z; v[3] = u0.w;
      v[4] = u1.x; v[5] = u1.y; v[6] = u1.z; v[7] = u1.w;
    } else if constexpr (sizeof(T) == 8) {
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const double2 u = __ldg(reinterpret_cast<const double2 *>(p) + h);
        v[2 * h] = u.x;
        v[2 * h + 1] = u.y;
      }
    } else {
      const uint4 u = __ldg(reinterpret_cast<const uint4 *>(p));
      const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        v[2 * h] = __ushort_as_bfloat16((unsigned short)(w[h] & 0xFFFFu));
        v[2 * h + 1] = __ushort_as_bfloat16((unsigned short)(w[h] >> 16));
      }
    }
  } else {
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int64_t lr = lr0 + t;
      v[t] = (j < a.n && lr >= 0 && lr < a.m) ? X[lr + (int64_t)j * a.ldx] : T(0);
    }
  }
}

// Writes the S slices of 8 consecutive rows of one column (bf16, 16 bytes per
// slice) to dst + b * slice_stride; slice b carries the multiple of 2^(-7b)
// of x 2^(6-e) described above.  e is the block's column exponent.
template <int PREC>
__device__ __forceinline__ void slice8_store(const typename SliceCfg<PREC>::T (&x)[8], int e, unsigned char *dst,
                                             int slice_stride) {
  constexpr int S = SliceCfg<PREC>::S;
  if constexpr (PREC == RCQR_F64) {
    unsigned long long F[8];
    uint32_t neg = 0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const unsigned long long bits = (unsigned long long)__double_as_longlong(x[t]);
      const int be = (int)((bits >> 52) & 0x7FF);
      neg |= (uint32_t)(bits >> 63) << t;
      unsigned long long f = 0;
      if ((bits << 1) != 0 && e != EMPTY_EXP) {
        // |x| = mant 2^(bx - 1075), with bx = 1 and no implicit bit for a subnormal x
        const unsigned long long frac = bits & 0xFFFFFFFFFFFFFull;
        const unsigned long long mant = be != 0 ? (frac | (1ull << 52)) : frac;
        const int d = e - ((be != 0 ? be : 1) - 1023);   // |x| < 2^(e+1): the shift keeps f below 2^56
        f = d <= 3 ? (mant << (3 - d)) : (d - 3 < 64 ? (mant >> (d - 3)) : 0ull);
      }
      F[t] = f;                                  // |x| 2^(55-e), below 2^56
    }
#pragma unroll
    for (int b = 0; b < S; ++b) {
      uint32_t w[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        float v[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int t = 2 * p + q;
          const uint32_t dig = (uint32_t)(F[t] >> (49 - 7 * b)) & 127u;
          float dv = __uint_as_float(0x4B000000u | dig) - 8388608.0f;   // the digit, exactly
          if (b > 0) dv *= pow2f(-7 * b);
          v[q] = ((neg >> t) & 1u) ? -dv : dv;
        }
        w[p] = __byte_perm(__float_as_uint(v[0]), __float_as_uint(v[1]), 0x7632);
      }
      *reinterpret_cast<uint4 *>(dst + b * slice_stride) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  } else {
    // FP32 / BF16 storage: t = x 2^(5-e) in (-64, 64); digit b = t rounded to a
    // multiple of 2^(-7b) by adding and removing 1.5 2^(23-7b); t -= digit (both
    // exact), so every digit is at most 64 in units of its slice.  Pairs of rows
    // go through the packed f32x2 unit.
    float t8[8];
    const int sh = 5 - e;
    const bool empty = e == EMPTY_EXP;
    const float s1 = empty ? 0.0f : pow2f(sh / 2), s2 = empty ? 0.0f : pow2f(sh - sh / 2);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      float x0, x1;
      if constexpr (PREC == RCQR_BF16) {
        x0 = __bfloat162float(x[2 * p]);
        x1 = __bfloat162float(x[2 * p + 1]);
      } else {
        x0 = x[2 * p];
        x1 = x[2 * p + 1];
      }
      mul2(x0, x1, x0, x1, s1, s1);
      mul2(t8[2 * p], t8[2 * p + 1], x0, x1, s2, s2);
    }
#pragma unroll
    for (int b = 0; b < S - 1; ++b) {
      const float M = __uint_as_float(((uint32_t)(150 - 7 * b) << 23) | 0x400000u);   // 1.5 2^(23-7b)
      uint32_t w[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        float u0, u1, d0, d1;
        add2(u0, u1, t8[2 * p], t8[2 * p + 1], M, M);
        add2(d0, d1, u0, u1, -M, -M);
        add2(t8[2 * p], t8[2 * p + 1], t8[2 * p], t8[2 * p + 1], -d0, -d1);
        w[p] = __byte_perm(__float_as_uint(d0), __float_as_uint(d1), 0x7632);
      }
      *reinterpret_cast<uint4 *>(dst + b * slice_stride) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    // the last slice feeds the shared (rounded) accumulator: the remainder itself,
    // rounded to bf16 (8 significant bits relative to the remainder)
    {
      uint32_t w[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(t8[2 * p], t8[2 * p + 1]);
        w[p] = *reinterpret_cast<const uint32_t *>(&h);
      }
      *reinterpret_cast<uint4 *>(dst + (S - 1) * slice_stride) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// The Theta tile of one stage: KCH * 128 rows of Theta x 32 rows of X, one
// Philox call per 16 X rows, spread over the NTW Theta warps (CPT calls per
// thread); each call's Theta row, 16-row sub-block and place in the tile are
// the same at every stage, so they are computed once.
template <int KCH, int NTW>
struct ThetaCalls {
  static constexpr int CPR = kBK / 16;                       // calls per Theta row and stage
  static constexpr int CPT = KCH * 128 * CPR / (32 * NTW);
  static_assert(CPT * 32 * NTW == KCH * 128 * CPR, "calls divide evenly");
  uint32_t row[CPT];   // Theta row i of the call (>= k: a zero row)
  uint32_t qq[CPT];    // 16-row sub-block within the stage
  uint32_t off[CPT];   // byte offset of the call's first 16 bytes in the tile

  __device__ __forceinline__ void init(int tt, int kgi) {
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      const int ci = tt + 32 * NTW * u;
      const int q = ci % CPR, r = ci / CPR;
      const int c = r >> 7, il = r & 127;
      row[u] = (uint32_t)((kgi * KCH + c) * 128 + il);
      qq[u] = (uint32_t)q;
      off[u] = (uint32_t)(c * (128 * kBK * 2) + (il >> 3) * (kBK * 16) + (il & 7) * 16 + 2 * q * 128);
    }
  }

  __device__ __forceinline__ void tile(unsigned char *sA, const uint32_t *tabp, int64_t r0, const TcArgs &a) const {
    const uint64_t qbase = (uint64_t)(r0 / 16);
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      uint32_t wv[8];
      if (row[u] < (uint32_t)a.k) {
        const uint64_t q = qbase + qq[u];
        const uint4 w = philox4x32_10_keys(make_uint4((uint32_t)q, (uint32_t)(q >> 32), row[u], a.stream_id), a.rk);
        const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          const uint32_t word = ww[p >> 1];
          const uint32_t b0 = __byte_perm(word, 0u, 0x4440u + 2u * (p & 1));
          const uint32_t b1 = __byte_perm(word, 0u, 0x4441u + 2u * (p & 1));
          wv[p] = __byte_perm(tabp[b0 << 5], tabp[b1 << 5], 0x5410);
        }
      } else {
#pragma unroll
        for (int p = 0; p < 8; ++p) wv[p] = 0u;
      }
      unsigned char *dst = sA + off[u];
      *reinterpret_cast<uint4 *>(dst) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
      *reinterpret_cast<uint4 *>(dst + 128) = make_uint4(wv[4], wv[5], wv[6], wv[7]);
    }
  }
};

// The Rademacher or SRHT Theta tile of one stage: thread tt (< KCH * 128) owns Theta row
// il = tt % 128 of chunk c = tt / 128 (row i = (kgi KCH + c) 128 + il).  Rademacher: its 32
// entries of the stage at global X rows r0 .. r0+31 are bits (r0 mod 128) .. +31 of the
// Philox call at counter (r0 / 128, i): one call per four stages, kept in registers.
// SRHT (Sec. 2, sqrt(1/k) S H D): the same bits of the call at counter (r0 / 128, 2^32 - 1)
// are the signs d_r, shared by every row, and entry (i, r) flips them by the parity of
// h_i AND r, h_i = the sampled Hadamard row (words 0, 1 of the call at counter
// (i, 0, 2^32 - 2)).  With r = r0 + j (r0 a multiple of 32, j < 32) that parity is
// parity(h_i AND r0) XOR parity(h_i AND j): one popcount per stage and a 32-bit mask of the
// second term computed once.  Bit 0 -> +1, 1 -> -1.
template <int KCH>
struct RadCalls {
  uint32_t row;     // Theta row i (>= k: a zero row)
  uint32_t off;     // byte offset of the row's first 16 bytes in the tile
  uint4 w;
  bool srht;
  uint64_t h;       // SRHT: the sampled Hadamard row
  uint32_t pmask;   // SRHT: bit j = parity(h AND j), j < 32

  __device__ __forceinline__ void init(int tt, int kgi, const TcArgs &a) {
    const int c = tt >> 7, il = tt & 127;
    row = (uint32_t)((kgi * KCH + c) * 128 + il);
    off = (uint32_t)(c * (128 * kBK * 2) + (il >> 3) * (kBK * 16) + (il & 7) * 16);
    w = make_uint4(0u, 0u, 0u, 0u);
    srht = a.dist == RCQR_THETA_SRHT;
    h = 0;
    pmask = 0;
    if (srht) {
      const uint4 hw = philox4x32_10_keys(make_uint4(row, 0u, 0xFFFFFFFEu, a.stream_id), a.rk);
      h = (uint64_t)hw.x | ((uint64_t)hw.y << 32);
      for (uint32_t j = 0; j < 32; ++j) pmask |= (uint32_t)(__popc((uint32_t)h & j) & 1) << j;
    }
  }

  __device__ __forceinline__ void tile(unsigned char *sA, int64_t r0, const TcArgs &a) {
    const int sub = (int)((r0 >> 5) & 3);          // the call's 32-bit word for these 32 rows
    if (sub == 0) {                                // stages start on 128-row boundaries at sub 0
      const uint64_t q = (uint64_t)(r0 >> 7);
      const uint32_t ctr = srht ? 0xFFFFFFFFu : row;
      w = (srht || row < (uint32_t)a.k)
              ? philox4x32_10_keys(make_uint4((uint32_t)q, (uint32_t)(q >> 32), ctr, a.stream_id), a.rk)
              : make_uint4(0u, 0u, 0u, 0u);
    }
    uint32_t word = sub == 0 ? w.x : (sub == 1 ? w.y : (sub == 2 ? w.z : w.w));
    if (srht) word ^= pmask ^ ((__popcll(h & (uint64_t)r0) & 1) ? 0xFFFFFFFFu : 0u);
    const bool live = row < (uint32_t)a.k;
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      uint32_t pv[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const uint32_t t = word >> (8 * kc + 2 * p);
        // bf16 +-1 pair: sign bits 15 and 31 from bits 0 and 1 of t
        pv[p] = live ? (0x3F803F80u | ((t << 15) & 0x8000u) | ((t << 30) & 0x80000000u)) : 0u;
      }
      *reinterpret_cast<uint4 *>(sA + off + kc * 128) = make_uint4(pv[0], pv[1], pv[2], pv[3]);
    }
  }
};

// Bounded mbarrier wait with growing sleeps between polls (a waiting warp
// leaves the issue slots to the working ones); gives up at once when another
// thread of the CTA has already timed out.
__device__ __forceinline__ void wait_or_fail(uint64_t *bar, uint32_t parity, int *fail, uint32_t max_sleep_ns,
                                             uint32_t polls) {
  volatile int *f = fail;
  uint32_t ns = 16;
  for (uint32_t round = 0; round < polls; ++round) {
    if (umma::mbar_wait(bar, parity, 1)) return;
    if (*f) return;
    __nanosleep(ns);
    ns = ns * 2 < max_sleep_ns ? ns * 2 : max_sleep_ns;
  }
  *f = 1;
}


template <int PREC, int KCH, int JCH>
struct Tc {
  using Cfg = SliceCfg<PREC>;
  using T = typename Cfg::T;
  using MaxT = typename Cfg::MaxT;
  static constexpr int S = Cfg::S, NE = Cfg::NE, LS = Cfg::LS;
  static constexpr int NACC = NE + 1;
  static constexpr int BR = block_rows(PREC);          // rows per block
  static constexpr int SPB = BR / kBK;                 // stages per block
  static constexpr int TOP = PREC == RCQR_F64 ? 6 : 5; // x = t 2^(e - TOP), t the scaled value sliced
  static constexpr int NC = 64 * JCH;                 // columns per CTA
  static constexpr int NTW = 4 * KCH;                 // Theta warps (two Philox calls per thread and stage)
  static constexpr int NXW = kProdWarps - NTW;        // X warps
  static constexpr uint32_t NCOLS = (KCH * NACC * NC) <= 256 ? 256u : 512u;
  static constexpr int A_BYTES = KCH * 128 * kBK * 2;
  static constexpr int B_BYTES = S * NC * kBK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static_assert(KCH * NACC * NC <= 512, "TMEM holds 512 columns");

  struct Shared {
    uint64_t full[kMaxStages];
    uint64_t empty[kMaxStages];
    uint64_t accf;
    uint64_t drain;      // completion of the MMA thread's last MMAs, before TMEM is released
    uint32_t tslot;
    int s_fail;
    int E_fix[NC];       // the int64 accumulators' column exponents: the largest block exponent of the CTA's rows
    int sft[NC];         // the folded block's right shift onto them (0 for an all-zero block column)
  };

  // Folds block b's TMEM accumulators into the int64 accumulators.  Run by all
  // 16 warps of the CTA (the producers join once they have filled the ring with
  // the next block's first stages: no further slot frees up before the fold has
  // read TMEM and the next MMAs run): warp w reads TMEM lanes 32 (w % 4) .. (its lane quadrant)
  // and takes every fourth 8-column chunk, starting at chunk w / 4; each thread
  // owns one Theta row of its chunks.  Starts and ends with a barrier of the
  // whole CTA, after which TMEM may be overwritten.
  static __device__ __noinline__ void fold(Shared &sh, int b, int NB, uint32_t tbase, long long *Acc,
                                           const TcArgs &a, int kgi, int col0, int g, int64_t blk) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lq = warp & 3, part = warp >> 2;
    const int il = 32 * lq + lane;
    // chunks of 8 columns; this thread's 8 accumulators of a chunk are contiguous,
    // Acc[(c 128 + il) NC + jl], and the next chunk's are loaded while this one is folded
    constexpr int CPC = NC / 8, NCH = KCH * CPC;
    auto acc_ptr = [&](int ch) {
      return reinterpret_cast<longlong2 *>(Acc + ((size_t)(ch / CPC) * 128 + il) * NC + (ch % CPC) * 8);
    };
    longlong2 nxt[4];
    if (b > 0 && part < NCH) {
#pragma unroll
      for (int h = 0; h < 4; ++h) nxt[h] = acc_ptr(part)[h];
    }
    const int *eb = a.eblk + (blk - a.blk0) * a.n;
    for (int jl = tid; jl < NC; jl += kThreadsTC) {
      const int e = col0 + jl < a.n ? __ldg(eb + col0 + jl) : EMPTY_EXP;
      const int d = sh.E_fix[jl] - e;
      sh.sft[jl] = e == EMPTY_EXP ? 0 : (d < 63 ? d : 63);
    }
    wait_or_fail(&sh.accf, (uint32_t)(b & 1), &sh.s_fail, 256, a.polls);
    umma::fence_after_sync();
    umma::named_sync(kThreadsTC);
    const bool last = b == NB - 1;
#pragma unroll 1
    for (int ch = part; ch < NCH; ch += 4) {
      const int c = ch / CPC, jc0 = (ch % CPC) * 8;
      const int i = (kgi * KCH + c) * 128 + il;
      longlong2 old2[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) old2[h] = nxt[h];
      if (b > 0 && ch + 4 < NCH) {
#pragma unroll
        for (int h = 0; h < 4; ++h) nxt[h] = acc_ptr(ch + 4)[h];
      }
      uint32_t rv[NACC][8];
#pragma unroll
      for (int acc = 0; acc < NACC; ++acc)
        umma::tmem_ld8(tbase + ((uint32_t)(32 * lq) << 16) + (uint32_t)((c * NACC + acc) * NC + jc0), rv[acc]);
      umma::tmem_wait_ld();
      long long out[8];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int jl = jc0 + jj;
        const long long old = b > 0 ? ((jj & 1) ? old2[jj >> 1].y : old2[jj >> 1].x) : 0LL;
        // the block's value in units of 2^(e - TOP - 7 NE - LS) (an all-zero block column
        // gives 0), then shifted onto the CTA's column exponent (floor, as the int64 sum)
        long long V = 0;
#pragma unroll
        for (int bs = 0; bs < NE; ++bs)
          V += (long long)__float2int_rn(__uint_as_float(rv[bs][jj]) * pow2f(7 * bs)) << (7 * (NE - bs) + LS);
        V += rint_to_ll(__uint_as_float(rv[NE][jj]) * pow2f(7 * NE + LS));   // |.| < 2^35
        const long long acc_v = old + (V >> sh.sft[jl]);
        out[jj] = acc_v;
        if (last) {
          const int j = col0 + jl;
          const int E = sh.E_fix[jl];
          if (i < a.k && j < a.n)
            a.partial[((int64_t)g * a.n + j) * a.k + i] = E == EMPTY_EXP ? 0.0 : ldexp((double)acc_v, E - TOP - 7 * NE - LS);
        }
      }
      if (!last) {
        longlong2 *ap = acc_ptr(ch);
#pragma unroll
        for (int h = 0; h < 4; ++h) ap[h] = make_longlong2(out[2 * h], out[2 * h + 1]);
      }
    }
    umma::fence_before_sync();
    umma::named_sync(kThreadsTC);
  }
};

// Asynchronous 16-byte global -> shared copy (no register staging).
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(umma::smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Column exponents of every block of br rows: eblk[(blk - blk0) * n + j], and
// (NORMS) the block's column sums of squares in FP64, ss[(blk - blk0) * n + j]
// -- the squared column norms of Sec. 4's normalisation come from the same
// pass over X.  One warp per (block, column), 8 per CTA; the rows outside
// [0, m) are skipped.
template <class T, bool NORMS>
__global__ void __launch_bounds__(256) block_exp_kernel(const T *__restrict__ X, int64_t m, int n, int64_t ldx,
                                                        int64_t row_offset, int64_t blk0, int64_t nblk, int br,
                                                        int *__restrict__ eblk, double *__restrict__ ss) {
  const int64_t w = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= nblk * n) return;
  const int64_t bl = w / n;
  const int j = (int)(w % n);
  const int64_t lr0 = (blk0 + bl) * br - row_offset;
  const T *col = X + (int64_t)j * ldx;
  decltype(mag_bits(T(0))) mx = 0;
  double s2 = 0.0;
  for (int r = lane; r < br; r += 32) {
    const int64_t lr = lr0 + r;
    if (lr >= 0 && lr < m) {
      const T v = __ldg(col + lr);
      mx = max(mx, mag_bits(v));
      if constexpr (NORMS) {
        const double d = to_f64(v);
        s2 = fma(d, d, s2);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) eblk[w] = block_exp(mx);
  if constexpr (NORMS) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (lane == 0) ss[w] = s2;
  }
}

// colnorm2[j] = sum over blocks of ss[b * n + j]: one warp per column, fixed order.
__global__ void block_norms_reduce_kernel(const double *__restrict__ ss, int64_t nblk, int n,
                                          double *__restrict__ colnorm2) {
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= n) return;
  const double s = warp_sum_strided(ss + j, (int)nblk, (int64_t)n);
  if ((threadIdx.x & 31) == 0) colnorm2[j] = s;
}

template <int PREC, int KCH, int JCH>
__global__ void __launch_bounds__(kThreadsTC, 1) sketch_tc_kernel(TcArgs a) {
  using K = Tc<PREC, KCH, JCH>;
  using T = typename K::T;
  constexpr int NC = K::NC, S = K::S;
  constexpr int NTW = K::NTW, NXW = K::NXW;
  constexpr int NTASK = 4 * NC;                        // (column, 8-row octet) pairs per stage
  constexpr int NXT = 32 * NXW;
  constexpr int TPT = NTASK / NXT;                     // tasks per X thread
  static_assert(TPT * NXT == NTASK, "X tasks divide evenly");
  constexpr int H = (int)(8 * sizeof(T) / 16);         // 16-byte chunks per octet
  constexpr int SLOT_BYTES = NTASK * 8 * (int)sizeof(T);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ typename K::Shared sh;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int D = a.D;
  const int g = blockIdx.y;
  const int kgi = blockIdx.x / a.ngrp, ngi = blockIdx.x % a.ngrp;
  const int col0 = ngi * NC;
  const T *X = static_cast<const T *>(a.X);
  uint32_t *table = reinterpret_cast<uint32_t *>(smem_raw);
  unsigned char *xring = smem_raw + kTableBytes;
  unsigned char *stage_base = xring + kXSlots * SLOT_BYTES;

  const int64_t bb = a.blk0 + (a.nblk * g) / a.groups;
  const int64_t be_ = a.blk0 + (a.nblk * (g + 1)) / a.groups;
  const int NB = (int)(be_ - bb);
  constexpr int kSPB = K::SPB, kBlockRows = K::BR;
  const int total = NB * kSPB;
  long long *Acc = a.acc64 + (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * (KCH * NC * 128);

  for (int e = tid; e < 256 * 32; e += kThreadsTC) {
    const int lev = (int)a.theta.level[e >> 5];
    table[e] = __float_as_uint((float)lev) >> 16;
  }
  for (int j = tid; j < NC; j += kThreadsTC) sh.E_fix[j] = EMPTY_EXP;
  if (tid == 0) {
    for (int s = 0; s < kMaxStages; ++s) {
      umma::mbar_init(&sh.full[s], kProdWarps);
      umma::mbar_init(&sh.empty[s], 1);
    }
    umma::mbar_init(&sh.accf, 1);
    umma::mbar_init(&sh.drain, 1);
    sh.s_fail = 0;
  }
  if (warp == 0) umma::tmem_alloc(&sh.tslot, K::NCOLS);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tbase = sh.tslot;
  {
    // column exponents of the int64 accumulators: the largest block exponent over the
    // CTA's blocks (fixed, so each block's value is shifted onto them once)
    static_assert(kThreadsTC % NC == 0, "whole columns per thread group");
    const int jl = tid % NC;
    if (col0 + jl < a.n) {
      int mx = EMPTY_EXP;
      for (int b = tid / NC; b < NB; b += kThreadsTC / NC) mx = max(mx, __ldg(a.eblk + (bb - a.blk0 + b) * a.n + col0 + jl));
      atomicMax(&sh.E_fix[jl], mx);
    }
  }
  __syncthreads();

  if (warp < NTW) {
    // ---- Theta producers
    const uint32_t *tabp = table + lane;
    ThetaCalls<KCH, NTW> calls;
    RadCalls<KCH> rad;
    const bool rademacher = a.dist != RCQR_THETA_GAUSSIAN;   // one bit per entry: Rademacher or SRHT
    if (rademacher) rad.init(tid, kgi, a);
    else calls.init(tid, kgi);
    // ring slot, its phase parity, block and stage within the block, first X row of
    // the stage: all advanced incrementally (blocks are contiguous, so the row is
    // bb BR + it kBK)
    int slot = 0, b = 0, st = 0;
    uint32_t ph = 0;
    int64_t r0 = bb * kBlockRows;
    for (int it = 0; it < total; ++it) {
      // the ring holds the next block's first D stages: fold the previous block (the
      // next slot is released only by MMAs issued after that fold)
      if (st == D && b > 0) K::fold(sh, b - 1, NB, tbase, Acc, a, kgi, col0, g, bb + b - 1);
      if (it >= D) wait_or_fail(&sh.empty[slot], ph ^ 1u, &sh.s_fail, 256, a.polls);
      if (rademacher) rad.tile(stage_base + slot * K::STAGE_BYTES, r0, a);
      else calls.tile(stage_base + slot * K::STAGE_BYTES, tabp, r0, a);
      umma::fence_proxy_async();
      __syncwarp();
      if (lane == 0) umma::mbar_arrive(&sh.full[slot]);
      r0 += kBK;
      if (++slot == D) { slot = 0; ph ^= 1u; }
      if (++st == kSPB) { st = 0; ++b; }
    }
    if (NB > 0) K::fold(sh, NB - 1, NB, tbase, Acc, a, kgi, col0, g, bb + NB - 1);
  } else if (warp < kProdWarps) {
    // ---- X producers: task o = xt + NXT u is column jl = 8 (o / 32) + o % 8, octet oc = (o / 8) % 4
    // (8 consecutive lanes: 8 consecutive columns of one octet, so the slice stores do not conflict)
    const int xt = tid - 32 * NTW;
    // per task: its column (j < n, else zeros), its 8-row octet, the row of that octet
    // in the CTA's first stage; a stage s adds s kBK rows (blocks are contiguous)
    static_assert((kXSlots & (kXSlots - 1)) == 0, "X ring slots: a power of two");
    const T *colp[TPT];
    int64_t lrb[TPT];
    bool fast[TPT];
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      const int o = xt + NXT * u;
      const int jl = 8 * (o >> 5) + (o & 7), oc = (o >> 3) & 3;
      const int j = col0 + jl;
      colp[u] = X + (int64_t)(j < a.n ? j : 0) * a.ldx;
      lrb[u] = bb * kBlockRows - a.row_offset + 8 * oc;
      fast[u] = j < a.n && a.vec;
    }
    // copies the octets of stage s into ring slot s mod kXSlots (asynchronously where possible)
    auto issue = [&](int s) {
      unsigned char *slot_base = xring + (s & (kXSlots - 1)) * SLOT_BYTES;
#pragma unroll
      for (int u = 0; u < TPT; ++u) {
        const int o = xt + NXT * u;
        const int64_t lr0 = lrb[u] + (int64_t)s * kBK;
        unsigned char *dst = slot_base + o * 16;
        if (fast[u] && lr0 >= 0 && lr0 + 8 <= a.m) {
          const unsigned char *src = reinterpret_cast<const unsigned char *>(colp[u] + lr0);
#pragma unroll
          for (int h = 0; h < H; ++h) cp_async16(dst + h * (NTASK * 16), src + 16 * h);
        } else {
          const int jl = 8 * (o >> 5) + (o & 7);
          __align__(16) T v[8];
          load8<T>(X, lr0, col0 + jl, a, v);
#pragma unroll
          for (int h = 0; h < H; ++h)
            *reinterpret_cast<uint4 *>(dst + h * (NTASK * 16)) = reinterpret_cast<const uint4 *>(v)[h];
        }
      }
    };
#pragma unroll 1
    for (int s = 0; s < kXAhead; ++s) {
      if (s < total) issue(s);
      cp_async_commit();
    }
    int e_cur[TPT], e_nxt[TPT];
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      const int o = xt + NXT * u;
      const int jl = 8 * (o >> 5) + (o & 7);
      e_cur[u] = col0 + jl < a.n ? a.eblk[(bb - a.blk0) * a.n + col0 + jl] : EMPTY_EXP;
      e_nxt[u] = e_cur[u];
    }
    int slot = 0, b = 0, st = 0;
    uint32_t ph = 0;
    for (int it = 0; it < total; ++it) {
      if (st == D && b > 0) K::fold(sh, b - 1, NB, tbase, Acc, a, kgi, col0, g, bb + b - 1);
      if (it + kXAhead < total) issue(it + kXAhead);
      cp_async_commit();
      if (st == kSPB / 2 && b + 1 < NB) {
        // exponents of the next block, read early
#pragma unroll
        for (int u = 0; u < TPT; ++u) {
          const int o = xt + NXT * u;
          const int jl = 8 * (o >> 5) + (o & 7);
          e_nxt[u] = col0 + jl < a.n ? a.eblk[(bb - a.blk0 + b + 1) * a.n + col0 + jl] : EMPTY_EXP;
        }
      }
      if (st == 0 && b > 0) {
#pragma unroll
        for (int u = 0; u < TPT; ++u) e_cur[u] = e_nxt[u];
      }
      cp_async_wait<kXAhead>();
      if (it >= D) wait_or_fail(&sh.empty[slot], ph ^ 1u, &sh.s_fail, 256, a.polls);
      unsigned char *sB = stage_base + slot * K::STAGE_BYTES + K::A_BYTES;
      const unsigned char *src = xring + (it & (kXSlots - 1)) * SLOT_BYTES;
#pragma unroll
      for (int u = 0; u < TPT; ++u) {
        const int o = xt + NXT * u;
        const int jl = 8 * (o >> 5) + (o & 7), oc = (o >> 3) & 3;
        __align__(16) T v[8];
#pragma unroll
        for (int h = 0; h < H; ++h)
          reinterpret_cast<uint4 *>(v)[h] = *reinterpret_cast<const uint4 *>(src + h * (NTASK * 16) + o * 16);
        slice8_store<PREC>(v, e_cur[u], sB + (jl >> 3) * (kBK * 16) + oc * 128 + (jl & 7) * 16, NC * kBK * 2);
      }
      umma::fence_proxy_async();
      __syncwarp();
      if (lane == 0) umma::mbar_arrive(&sh.full[slot]);
      if (++slot == D) { slot = 0; ph ^= 1u; }
      if (++st == kSPB) { st = 0; ++b; }
    }
    cp_async_wait<0>();
    if (NB > 0) K::fold(sh, NB - 1, NB, tbase, Acc, a, kgi, col0, g, bb + NB - 1);
  } else if (warp < kThreadsTC / 32 - 1) {
    // ---- warps 12..14: fold only
    for (int b = 0; b < NB; ++b) K::fold(sh, b, NB, tbase, Acc, a, kgi, col0, g, bb + b);
  } else {
    // ---- warp 15: one thread issues the MMAs; after a block's last stage the warp folds with the others.
    // Slices 0..NE feed consecutive accumulators and sit consecutively in the
    // stage, so up to 256 / NC of them form one MMA with N = (count) NC (the
    // Theta tile is then read once for all of them); the slices below NE add
    // into accumulator NE one MMA each.
    constexpr int G = 256 / NC;
    // operand descriptors of ring slot 0; a slot, chunk, K step or slice adds its byte
    // offset / 16 to the start-address field (shared addresses stay below 2^18 bytes,
    // so the 14-bit field does not carry)
    const uint64_t desc0 = umma::smem_desc(umma::smem_u32(stage_base), 128, kBK * 16);
    int slot = 0, b = 0, st = 0;
    uint32_t ph = 0;
    for (int it = 0; it < total; ++it) {
      // once any wait of the CTA has given up, no further MMA is issued (the partial sums
      // become NaN below), so nothing new is in flight when TMEM is released
      if (lane == 0) wait_or_fail(&sh.full[slot], ph, &sh.s_fail, 64, a.polls);
      if (lane == 0 && *(volatile int *)&sh.s_fail == 0) {
        umma::fence_after_sync();
        const uint64_t dslot = desc0 + (uint64_t)((slot * K::STAGE_BYTES) >> 4);
#pragma unroll
        for (int c = 0; c < KCH; ++c)
#pragma unroll
          for (int q = 0; q < kBK / 16; ++q) {
            const uint64_t ad = dslot + (uint64_t)((c * (128 * kBK * 2) + q * 256) >> 4);
            const bool first = (st == 0) && (q == 0);
#pragma unroll
            for (int g0 = 0; g0 <= K::NE; g0 += G) {
              const int cnt = (K::NE + 1 - g0) < G ? (K::NE + 1 - g0) : G;
              const uint32_t dcol = tbase + (uint32_t)((c * K::NACC + g0) * NC);
              const uint64_t bd = dslot + (uint64_t)((K::A_BYTES + g0 * (NC * kBK * 2) + q * 256) >> 4);
              umma::mma_bf16(dcol, ad, bd, umma::idesc_bf16_f32(128, cnt * NC), first ? 0u : 1u);
            }
#pragma unroll
            for (int bs = K::NE + 1; bs < S; ++bs) {
              const uint32_t dcol = tbase + (uint32_t)((c * K::NACC + K::NE) * NC);
              const uint64_t bd = dslot + (uint64_t)((K::A_BYTES + bs * (NC * kBK * 2) + q * 256) >> 4);
              umma::mma_bf16(dcol, ad, bd, umma::idesc_bf16_f32(128, NC), 1u);
            }
          }
        umma::mma_commit(&sh.empty[slot]);
        if (st == kSPB - 1) umma::mma_commit(&sh.accf);
      }
      __syncwarp();
      if (st == kSPB - 1) K::fold(sh, b, NB, tbase, Acc, a, kgi, col0, g, bb + b);
      if (++slot == D) { slot = 0; ph ^= 1u; }
      if (++st == kSPB) { st = 0; ++b; }
    }
    // drain: the barrier completes once every MMA this thread issued has finished
    // writing TMEM (at once if none was issued); bounded by the default limit, so a
    // shortened test limit cannot release TMEM under a running MMA
    if (lane == 0) {
      umma::mma_commit(&sh.drain);
      if (!umma::mbar_wait(&sh.drain, 0u, kWaitPolls)) sh.s_fail = 1;
    }
    __syncwarp();
  }

  // every thread is done: the last fold consumed the last MMAs and read TMEM
  __syncthreads();
  if (*(volatile int *)&sh.s_fail != 0) {
    for (int e = tid; e < KCH * 128 * NC; e += kThreadsTC) {
      const int il = e % (KCH * 128), jl = e / (KCH * 128);
      const int i = kgi * KCH * 128 + il, j = col0 + jl;
      if (i < a.k && j < a.n) a.partial[((int64_t)g * a.n + j) * a.k + i] = __longlong_as_double(0x7FF8000000000000ll);
    }
    if (tid == 0 && a.status && atomicCAS(a.status, 0, (int)RCQR_ETIMEOUT) == 0) a.status[1] = -1;
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tbase, K::NCOLS);
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
  int JCH, NC, ngrp, KCH, kgrp, D, groups, S, BR;
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
  // as many 32-row stages as fit beside the level table and the X copy ring (at most kMaxStages)
  const size_t stage = (size_t)p.KCH * 128 * kBK * 2 + (size_t)p.S * p.NC * kBK * 2;
  const size_t ring = (size_t)kXSlots * 4 * p.NC * 8 * elem_size(prec);
  const size_t budget = 220 * 1024 - kTableBytes - ring;
  p.D = (int)std::min<size_t>(kMaxStages, budget / stage);
  p.smem = kTableBytes + ring + (size_t)p.D * stage;
  p.BR = block_rows(prec);
  p.blk0 = row_offset / p.BR;
  p.nblk = (row_offset + m + p.BR - 1) / p.BR - p.blk0;
  // row groups: one wave of CTAs (one per SM) when every CTA can take its share of
  // the blocks (at most maxb, the int64 headroom); otherwise as many groups as fill
  // whole waves, so the last wave is not a partial one
  const int64_t ctas_per_rows = (int64_t)p.kgrp * p.ngrp;
  const int64_t sms = num_sms();
  const int64_t gmin = (p.nblk + maxb - 1) / maxb;
  int64_t groups = std::min<int64_t>(std::max<int64_t>(1, sms / ctas_per_rows), p.nblk);
  if (groups < gmin) {
    const int64_t waves = (gmin * ctas_per_rows + sms - 1) / sms;
    groups = std::min<int64_t>(std::max<int64_t>(gmin, waves * sms / ctas_per_rows), p.nblk);
  }
  p.groups = (int)std::min<int64_t>(groups, 65535);
  return p;
}

size_t acc64_count(const TcPlan &p) {
  return (size_t)p.groups * p.kgrp * p.ngrp * p.KCH * p.NC * 128;
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

namespace {
std::atomic<uint32_t> g_wait_polls{kWaitPolls};
}  // namespace

uint32_t wait_polls() { return g_wait_polls.load(std::memory_order_relaxed); }

uint32_t set_wait_polls(uint32_t polls) {
  return g_wait_polls.exchange(polls == 0 ? kWaitPolls : polls, std::memory_order_relaxed);
}

bool sketch_tc_supported(int64_t n, int64_t k) {
  (void)k;
  return n >= 1 && n <= 256;
}

size_t sketch_tc_workspace(int64_t m, int64_t n, int64_t k, int64_t row_offset, int prec) {
  const TcPlan p = plan_tc(m, n, k, row_offset, prec);
  Workspace w(nullptr, 0);
  w.take<double>((size_t)p.groups * n * k);
  w.take<long long>(acc64_count(p));
  w.take<int>((size_t)p.nblk * n);
  w.take<double>((size_t)p.nblk * n);
  return w.used;
}

cudaError_t launch_sketch_tc(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, int64_t k,
                             uint64_t seed, uint32_t stream_id, int64_t row_offset, double *P,
                             int64_t ldp, double *colnorm2, int *dev_status, Workspace &ws, cudaStream_t st,
                             int dist) {
  const TcPlan p = plan_tc(m, n, k, row_offset, prec);
  double *partial = ws.take<double>((size_t)p.groups * n * k);
  long long *acc64 = ws.take<long long>(acc64_count(p));
  int *eblk = ws.take<int>((size_t)p.nblk * n);
  double *ss = ws.take<double>((size_t)p.nblk * n);
  if (!partial || !acc64 || !eblk || !ss) return cudaErrorMemoryAllocation;
  TcArgs a;
  a.X = X;
  a.m = m;
  a.n = (int)n;
  a.ldx = ldx;
  a.k = (int)k;
  a.seed = seed;
  a.stream_id = stream_id;
  for (int r = 0; r < 10; ++r) {
    a.rk[2 * r] = (uint32_t)seed + (uint32_t)r * 0x9E3779B9u;
    a.rk[2 * r + 1] = (uint32_t)(seed >> 32) + (uint32_t)r * 0xBB67AE85u;
  }
  a.row_offset = row_offset;
  a.blk0 = p.blk0;
  a.nblk = p.nblk;
  a.groups = p.groups;
  a.ngrp = p.ngrp;
  a.D = p.D;
  const size_t es = elem_size(prec);
  a.vec = ((uintptr_t)X % 16 == 0) && ((size_t)ldx * es) % 16 == 0 && ((size_t)row_offset * es) % 16 == 0;
  a.partial = partial;
  a.acc64 = acc64;
  a.eblk = eblk;
  a.status = dev_status;
  a.polls = wait_polls();
  a.theta = theta_table();
  a.dist = dist;
  dim3 grid((unsigned)(p.kgrp * p.ngrp), (unsigned)p.groups);
  cudaError_t e;
  {
    const unsigned eg = (unsigned)((p.nblk * n + 7) / 8);
#define RCQR_BEXP(TT)                                                                                             \
  if (colnorm2)                                                                                                   \
    block_exp_kernel<TT, true><<<eg, 256, 0, st>>>((const TT *)X, m, (int)n, ldx, row_offset, p.blk0, p.nblk, p.BR, \
                                                   eblk, ss);                                                    \
  else                                                                                                            \
    block_exp_kernel<TT, false><<<eg, 256, 0, st>>>((const TT *)X, m, (int)n, ldx, row_offset, p.blk0, p.nblk,      \
                                                    p.BR, eblk, nullptr);
    switch (prec) {
      case RCQR_F64: RCQR_BEXP(double) break;
      case RCQR_F32: RCQR_BEXP(float) break;
      default: RCQR_BEXP(__nv_bfloat16)
    }
#undef RCQR_BEXP
    if (colnorm2)
      block_norms_reduce_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(ss, p.nblk, (int)n, colnorm2);
  }
  switch (prec) {
    case RCQR_F64: e = launch_tc_prec<RCQR_F64>(a, p, grid, st); break;
    case RCQR_F32: e = launch_tc_prec<RCQR_F32>(a, p, grid, st); break;
    default: e = launch_tc_prec<RCQR_BF16>(a, p, grid, st);
  }
  if (e != cudaSuccess) return e;
  const double c = dist != RCQR_THETA_GAUSSIAN ? 1.0 / std::sqrt((double)k) : theta_scale(k);
  sketch_tc_reduce_kernel<<<(unsigned)((k * n * 32 + 255) / 256), 256, 0, st>>>(partial, p.groups, (int)k, (int)n,
                                                                          c, P, ldp);
  return cudaGetLastError();
}

}  // namespace rcqr
