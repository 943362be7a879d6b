// Q = X R^{-1} (Alg. 2 step 3; Alg. 7 step 4 with a permutation and a rank) for
// 64 < n <= 128 on FP32 / BF16 X: a blocked substitution with the off-diagonal
// products on the tcgen05 tensor cores.
//
// A CTA of 128 threads takes tiles of 128 rows (thread t owns row t of the tile and
// TMEM lane t).  The 128 (padded) columns form eight blocks of 16.  For block J the
// thread forms y_J = x_J - (sum_{I<J} q_I R_{I,J}) and solves y_J = q_J R_{J,J} by
// substitution in FP32 registers (R_{J,J} rounded to FP32, its diagonal as FP32
// reciprocals; the diagonal block is never inverted).  Right-looking: once block J is
// solved, q_J is split exactly into three bf16 pieces (h + m + l = q, each 8 significant
// bits, RN) into a 16-column operand buffer, and one group of MMAs adds q_J R_{J,>J} into
// the FP32 TMEM accumulator of the later columns.  R (FP32) is split the same way; the
// six products with piece indices summing to at most two are kept (the dropped ones are
// below 2^-26 of |q||R|), so each update carries the error of an FP32 sum of products
// and the row-wise backward error stays that of an FP32 substitution,
// Q (R + dR) = X with |dR| <= c n u |R|, u = 2^-24 (Higham Thm. 8.5).
//
// Only the blocks R_{J,>J} are ever read by the MMAs, so the three pieces of R are kept
// in triangular regions: region J (rows 16J .. 16J+15 of R, the K dimension of block
// J's update) holds columns 16(J+1) .. 127 only, as K-major core matrices (two along K,
// 8-column groups 256 bytes apart).  The accumulator's TMEM column c is output column
// c + 16.
#include <algorithm>

#include "common.cuh"
#include "rcqr_internal.h"
#include "umma.cuh"

namespace rcqr {

namespace {

constexpr int kWR = 128;                       // rows per tile = TMEM lanes = threads
constexpr int kWN = 128;                       // padded columns
constexpr int kWB = kWN / 16;                  // blocks of 16 columns
constexpr uint32_t kWQSBO = (48 / 8) * 128;    // q piece buffer: K extent 48 (3 pieces x 16)
constexpr int kWQBytes = kWR * 48 * 2;         // 12 KB
constexpr uint32_t kWaitRoundsW = 1u << 20;    // bounded waits: rounds of try_wait (<= 1 us each)

// start of region J of one R piece, and the piece's size
__host__ __device__ constexpr uint32_t r_region(int J) { return 32u * (uint32_t)(J * (kWN - 16) - 16 * J * (J - 1) / 2); }
constexpr int kWRPiece = (int)r_region(kWB - 1);   // regions 0 .. kWB-2 (the last block has no update)
// element (output column j >= 16 (J+1), K row i of block J = i / 16) of one R piece
__host__ __device__ constexpr uint32_t r_offset(int j, int i) {
  const int J = i / 16;
  return r_region(J) + (uint32_t)((j - 16 * (J + 1)) / 8) * 256u + (uint32_t)((i % 16) / 8) * 128u +
         (uint32_t)(j % 8) * 16u + (uint32_t)(i % 8) * 2u;
}

constexpr int OFF_R = kWQBytes;
constexpr int OFF_RD = OFF_R + 3 * kWRPiece;            // diagonal blocks, kWB x 16 x 16 floats
constexpr int OFF_DS = OFF_RD + kWB * 256 * 4;          // fl32(1 / R_jj)
constexpr int OFF_SRC = OFF_DS + kWN * 4;               // source column of X per column
constexpr int kWSmem = OFF_SRC + kWN * 4;
// BF16 X: the tile is staged in shared memory (column c of the tile at bytes 256 c),
// copied in 16-byte pieces while the previous tile is solved: the threads' own 2-byte
// loads of a row along the columns used half of every memory transaction
constexpr int OFF_XS = kWSmem;
constexpr int kWSmemBf16 = OFF_XS + kWR * kWN * 2;
constexpr int kWCtas = 2;
static_assert(kWCtas * (kWSmemBf16 + 2048) <= 228 * 1024, "CTAs per SM");

__device__ __forceinline__ void cp_async16w(void *dst, const void *src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(umma::smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}

struct TcwArgs {
  const void *X;
  int64_t m;
  int n;
  int64_t ldx;
  const float *Rf;      // 128 x 128 FP32, column-major, zero beyond the rank (trsm32_prep_kernel)
  const float *dinv;    // fl32(1 / R_jj), 0 beyond the rank
  const int32_t *perm;  // nullable
  const int64_t *rank;  // nullable
  float *Q;
  int64_t ldq;
  int *status;          // nullable: RCQR_ETIMEOUT on a wait that gave up
  int vec;              // BF16 X: rows 16-byte aligned (the staged copy uses 16-byte pieces)
};

__device__ __forceinline__ float to_f32w(float x) { return x; }
__device__ __forceinline__ float to_f32w(__nv_bfloat16 x) { return __bfloat162float(x); }

// Exact three-way bf16 split of two FP32 values: x = h + m + l for each.
__device__ __forceinline__ void split3w(float x0, float x1, uint32_t &h, uint32_t &mm, uint32_t &l) {
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

__device__ __forceinline__ bool wait_upd(uint64_t *bar, uint32_t parity, int *fail) {
  for (uint32_t it = 0; it < kWaitRoundsW; ++it) {
    if (*(volatile int *)fail) return false;
    if (umma::mbar_try_wait_hint(bar, parity, 1000)) return true;
  }
  *(volatile int *)fail = 1;
  return false;
}

template <class TX>
__global__ void __launch_bounds__(kWR, kWCtas) trsm_tcw_kernel(TcwArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *Qs = smem;                                      // q_J pieces, K-major core matrices
  unsigned char *Rs = smem + OFF_R;                              // 3 triangular pieces of R
  float *Rd = reinterpret_cast<float *>(smem + OFF_RD);          // Rd[J][c][i] = R_{16J+i, 16J+c}
  float *Ds = reinterpret_cast<float *>(smem + OFF_DS);
  int *Src = reinterpret_cast<int *>(smem + OFF_SRC);
  __shared__ uint64_t bar_upd, bar_drain;
  __shared__ uint32_t tslot;
  __shared__ int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5;
  const TX *X = static_cast<const TX *>(a.X);
  const int r = a.rank ? (int)(*a.rank < (int64_t)a.n ? *a.rank : (int64_t)a.n) : a.n;

  // ---- set-up: the pieces of R's off-diagonal blocks, its diagonal blocks, 1 / R_jj
  for (int e = tid; e < kWN * kWN / 2; e += kWR) {
    const int j = e / (kWN / 2), i = 2 * (e % (kWN / 2));   // rows i, i+1 of column j
    if (j < 16 * (i / 16 + 1)) continue;                     // not in an off-diagonal block
    uint32_t h, mm, l;
    split3w(a.Rf[i + j * kWN], a.Rf[i + 1 + j * kWN], h, mm, l);
    const uint32_t off = r_offset(j, i);
    *reinterpret_cast<uint32_t *>(Rs + off) = h;
    *reinterpret_cast<uint32_t *>(Rs + kWRPiece + off) = mm;
    *reinterpret_cast<uint32_t *>(Rs + 2 * kWRPiece + off) = l;
  }
  for (int e = tid; e < kWB * 256; e += kWR) {
    const int J = e >> 8, c = (e >> 4) & 15, i = e & 15;
    Rd[e] = a.Rf[(16 * J + i) + (16 * J + c) * kWN];
  }
  for (int j = tid; j < kWN; j += kWR) {
    Ds[j] = a.dinv[j];
    Src[j] = j < r ? (a.perm ? a.perm[j] : j) : -1;
  }
  if (tid == 0) {
    umma::mbar_init(&bar_upd, 1);
    umma::mbar_init(&bar_drain, 1);
    s_fail = 0;
  }
  if (warp == 0) umma::tmem_alloc(&tslot, 128u);
  umma::fence_proxy_async();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tbase = tslot;
  const uint32_t lane_base = tbase + ((uint32_t)(32 * warp) << 16);
  const uint32_t qs_addr = umma::smem_u32(Qs), rs_addr = umma::smem_u32(Rs);
  const uint32_t row_sw = (uint32_t)(tid / 8) * kWQSBO + (uint32_t)(tid % 8) * 16;   // this row's core offset
  const int n = a.n;
  uint32_t ph = 0;

  const int64_t tiles = (a.m + kWR - 1) / kWR;
  constexpr bool kStage = sizeof(TX) == 2;
  __nv_bfloat16 *Xs = reinterpret_cast<__nv_bfloat16 *>(smem + OFF_XS);
  // BF16: copies tile tl (its columns in Src order) into Xs, rows past m read as zero
  auto stage = [&](int64_t tl) {
    const int64_t r0 = tl * kWR;
    for (int e = tid; e < kWN * (kWR / 8); e += kWR) {
      const int c = e / (kWR / 8), q8 = e % (kWR / 8);
      const int src = Src[c];
      if (src < 0) continue;
      const int64_t rw = r0 + 8 * q8;
      const int64_t left = a.m - rw;
      const int valid = left > 0 ? (int)(left < 8 ? left : 8) : 0;
      const TX *g = X + rw + (int64_t)src * a.ldx;
      cp_async16w(Xs + c * kWR + 8 * q8, valid > 0 ? (const void *)g : (const void *)X, 2 * valid);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if (kStage && a.vec && (int64_t)blockIdx.x < tiles) stage(blockIdx.x);
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t row = tile * kWR + tid;
    const bool live = row < a.m;
    float q[kWN];
    if (kStage && a.vec) {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      __syncthreads();
#pragma unroll
      for (int j = 0; j < kWN; ++j) q[j] = (live && Src[j] >= 0) ? __bfloat162float(Xs[j * kWR + tid]) : 0.0f;
      __syncthreads();                                   // Xs read by every thread: copy the next tile
      if (tile + gridDim.x < tiles) stage(tile + gridDim.x);
    } else {
#pragma unroll
      for (int j = 0; j < kWN; ++j) {
        const int src = Src[j];
        q[j] = (live && src >= 0) ? to_f32w(X[row + (int64_t)src * a.ldx]) : 0.0f;
      }
    }
#pragma unroll
    for (int J = 0; J < kWB; ++J) {
      if (J > 0) {
        // y_J = x_J - (the tensor-core sum of the earlier blocks' products)
        wait_upd(&bar_upd, ph, &s_fail);
        ph ^= 1u;
        umma::fence_after_sync();
        uint32_t v[16];
        umma::tmem_ld16(lane_base + 16 * (J - 1), v);
        umma::tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 16; ++c) q[16 * J + c] -= __uint_as_float(v[c]);
      }
      // substitution against the diagonal block R_{J,J} (column c: 16 floats at rd + 16 c),
      // each dot product in two interleaved FMA chains
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
      if (J < kWB - 1) {
        // the exact three-way split of q_J (two 16-byte chunks per piece); the previous
        // block's MMAs, the last readers of this buffer, completed before its update above
#pragma unroll
        for (int h8 = 0; h8 < 2; ++h8) {
          uint32_t hw[4], mw[4], lw[4];
#pragma unroll
          for (int p = 0; p < 4; ++p)
            split3w(q[16 * J + 8 * h8 + 2 * p], q[16 * J + 8 * h8 + 2 * p + 1], hw[p], mw[p], lw[p]);
          *reinterpret_cast<uint4 *>(Qs + row_sw + ((0 + 8 * h8) / 8) * 128) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          *reinterpret_cast<uint4 *>(Qs + row_sw + ((16 + 8 * h8) / 8) * 128) = make_uint4(mw[0], mw[1], mw[2], mw[3]);
          *reinterpret_cast<uint4 *>(Qs + row_sw + ((32 + 8 * h8) / 8) * 128) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        umma::fence_proxy_async();
        umma::fence_before_sync();
        __syncthreads();
        if (tid == 0 && !*(volatile int *)&s_fail) {
          umma::fence_after_sync();
          const int N = kWN - 16 * (J + 1);
          const uint32_t id = umma::idesc_bf16_f32(kWR, N);
          // (q piece, R piece) pairs with index sum <= 2
          const int pa[6] = {0, 0, 1, 0, 1, 2}, pr[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
          for (int p = 0; p < 6; ++p) {
            const uint64_t ad = umma::smem_desc(qs_addr + (uint32_t)((16 * pa[p]) / 8) * 128, 128, kWQSBO);
            const uint64_t bd = umma::smem_desc(rs_addr + (uint32_t)(pr[p] * kWRPiece) + r_region(J), 128, 256);
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
      for (int j = 0; j < kWN; ++j)
        if (j < n) a.Q[row + (int64_t)j * ldq] = q[j];
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
  if (warp == 0) umma::tmem_dealloc(tbase, 128u);
}

}  // namespace

bool trsm_tcw_supported(int64_t n) { return n > 64 && n <= 128; }

cudaError_t launch_trsm_tcw(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, const float *Rf,
                            const float *dinv, const int32_t *perm, const int64_t *rank, float *Q, int64_t ldq,
                            int *status, cudaStream_t st) {
  const int vec = ((uintptr_t)X % 16 == 0) && (ldx % 8 == 0);
  TcwArgs a{X, m, (int)n, ldx, Rf, dinv, perm, rank, Q, ldq, status, vec};
  const int64_t tiles = (m + kWR - 1) / kWR;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)kWCtas * num_sms()));
  cudaError_t e;
  if (prec == RCQR_BF16) {
    if ((e = set_smem(trsm_tcw_kernel<__nv_bfloat16>, kWSmemBf16)) != cudaSuccess) return e;
    trsm_tcw_kernel<__nv_bfloat16><<<grid, kWR, kWSmemBf16, st>>>(a);
  } else {
    if ((e = set_smem(trsm_tcw_kernel<float>, kWSmem)) != cudaSuccess) return e;
    trsm_tcw_kernel<float><<<grid, kWR, kWSmem, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace rcqr
