// Sketch P = Theta X (Alg. 2 step 1) on CUDA cores with FP64 accumulation (the
// kernel behind rcqr_sketch_noalloc), the squared column norms, the dense left
// product Y = L X of the reduced variant, and the entry of the factorization
// path's sketch, which runs the exact tensor-core kernel of sketch_tc.cu.
//
// Split-K over the long dimension m: CTA (chunk, g) walks a contiguous range
// of 64-row tiles of X (tiles aligned to multiples of 64 in *global* row
// space, so any row_offset works), generates the matching 64 x 64 block of
// Theta's integer levels in shared memory from Philox, and accumulates a
// 64 x 32 block of P in FP64 registers.  Partial sketches go to the workspace
// and a second kernel adds them in a fixed order (the "simple addition"
// reduction of Sec. 3.1) and applies the scale 1/sqrt(k v) in FP64.
// The same file holds the squared column norms (matrix D of Sec. 4) and the
// dense left product Y = L X of the reduced variant (Alg. 5 step 1).
#include <algorithm>

#include "common.cuh"
#include "rcqr_internal.h"
#include "theta.cuh"

namespace rcqr {

namespace {

constexpr int kTileRows = 64;  // rows of X per tile
constexpr int kChunkK = 64;    // rows of Theta per CTA
constexpr int kChunkN = 32;    // columns of X per CTA
constexpr int kThreads = 256;
constexpr int kLRows = 32;     // rows per tile of the dense left product

template <class TX>
__global__ void __launch_bounds__(kThreads)
sketch_partial_kernel(const TX *__restrict__ X, int64_t m, int n, int64_t ldx, int k,
                      uint64_t seed, uint32_t stream_id, int64_t row_offset, int64_t tile0,
                      int64_t ntiles, int groups, ThetaTable table, double *__restrict__ partial) {
  __shared__ float th[kChunkK][kTileRows + 1];  // integer levels, exact in float
  __shared__ double xs[kTileRows][kChunkN];
  __shared__ int8_t lev[256];

  const int nchunk_n = (n + kChunkN - 1) / kChunkN;
  const int kc0 = (blockIdx.x / nchunk_n) * kChunkK;
  const int nc0 = (blockIdx.x % nchunk_n) * kChunkN;
  const int g = blockIdx.y;
  const int tid = threadIdx.x;
  if (tid < 256) lev[tid] = table.level[tid];

  const int64_t tb = tile0 + (ntiles * g) / groups;
  const int64_t te = tile0 + (ntiles * (g + 1)) / groups;

  const int lane_j = tid & 31;      // output column within the chunk
  const int ibase = (tid >> 5) * 8;  // 8 output rows per thread
  double acc[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) acc[u] = 0.0;

  for (int64_t t = tb; t < te; ++t) {
    const int64_t grow0 = t * kTileRows;  // global row of the tile's first row
    __syncthreads();
    {  // Theta levels: thread -> (row i, 16-row block qb)
      const int il = tid >> 2, qb = tid & 3;
      const int i = kc0 + il;
      if (i < k) {
        const uint4 w = theta_block((uint64_t)(grow0 / 16 + qb), (uint32_t)i, stream_id, seed);
#pragma unroll
        for (int b = 0; b < 16; ++b) th[il][qb * 16 + b] = (float)lev[byte_of(w, b)];
      } else {
#pragma unroll
        for (int b = 0; b < 16; ++b) th[il][qb * 16 + b] = 0.0f;
      }
    }
    {  // X tile (zero outside [0, m) and beyond column n)
      const int r = tid & 63;
      const int64_t lr = grow0 + r - row_offset;
#pragma unroll
      for (int it = 0; it < kChunkN / 4; ++it) {
        const int jj = (tid >> 6) + 4 * it;
        const int j = nc0 + jj;
        double v = 0.0;
        if (lr >= 0 && lr < m && j < n) v = to_f64(X[lr + (int64_t)j * ldx]);
        xs[r][jj] = v;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < kTileRows; ++r) {
      const double xv = xs[r][lane_j];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] = fma((double)th[ibase + u][r], xv, acc[u]);
    }
  }
  const int j = nc0 + lane_j;
  if (j < n) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = kc0 + ibase + u;
      if (i < k) partial[((int64_t)g * n + j) * k + i] = acc[u];
    }
  }
}

// P(i, j) = c * sum_g partial[g](i, j), g in increasing order.
__global__ void sketch_reduce_kernel(const double *__restrict__ partial, int groups, int k, int n,
                                     double c, double *__restrict__ P, int64_t ldp) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)k * n) return;
  const int i = (int)(idx % k), j = (int)(idx / k);
  double s = 0.0;
  for (int g = 0; g < groups; ++g) s += partial[((int64_t)g * n + j) * k + i];
  P[i + (int64_t)j * ldp] = c * s;
}

// Partial squared column norms: CTA g sums rows [g*m/G, (g+1)*m/G) of every column.
template <class TX>
__global__ void colnorm_partial_kernel(const TX *__restrict__ X, int64_t m, int n, int64_t ldx,
                                       int groups, double *__restrict__ partial) {
  __shared__ double red[32];
  const int g = blockIdx.x;
  const int64_t rb = (m * g) / groups, re = (m * (g + 1)) / groups;
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int64_t r = rb + threadIdx.x; r < re; r += blockDim.x) {
      const double v = to_f64(X[r + (int64_t)j * ldx]);
      s = fma(v, v, s);
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) partial[(int64_t)g * n + j] = s;
  }
}

__global__ void colnorm_reduce_kernel(const double *__restrict__ partial, int groups, int n,
                                      double *__restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int g = 0; g < groups; ++g) s += partial[(int64_t)g * n + j];
  out[j] = s;
}

// Y = L X partials: same structure as the sketch with L read from memory.
template <class TX>
__global__ void __launch_bounds__(kThreads)
dense_left_partial_kernel(const double *__restrict__ L, int l, int64_t ldl, const TX *__restrict__ X,
                          int64_t m, int n, int64_t ldx, int groups, double *__restrict__ partial) {
  __shared__ double th[kChunkK][kLRows + 1];
  __shared__ double xs[kLRows][kChunkN];
  const int nchunk_n = (n + kChunkN - 1) / kChunkN;
  const int kc0 = (blockIdx.x / nchunk_n) * kChunkK;
  const int nc0 = (blockIdx.x % nchunk_n) * kChunkN;
  const int g = blockIdx.y;
  const int tid = threadIdx.x;
  const int64_t ntiles = (m + kLRows - 1) / kLRows;
  const int64_t tb = (ntiles * g) / groups, te = (ntiles * (g + 1)) / groups;
  const int lane_j = tid & 31, ibase = (tid >> 5) * 8;
  double acc[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) acc[u] = 0.0;
  for (int64_t t = tb; t < te; ++t) {
    const int64_t r0 = t * kLRows;
    __syncthreads();
    for (int e = tid; e < kChunkK * kLRows; e += kThreads) {
      const int il = e / kLRows, r = e % kLRows;
      const int i = kc0 + il;
      const int64_t lr = r0 + r;
      th[il][r] = (i < l && lr < m) ? L[i + lr * ldl] : 0.0;
    }
    {
      const int r = tid & (kLRows - 1);
      const int64_t lr = r0 + r;
#pragma unroll
      for (int it = 0; it < kChunkN / 8; ++it) {
        const int jj = (tid / kLRows) + 8 * it;
        const int j = nc0 + jj;
        xs[r][jj] = (lr < m && j < n) ? to_f64(X[lr + (int64_t)j * ldx]) : 0.0;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < kLRows; ++r) {
      const double xv = xs[r][lane_j];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] = fma((double)th[ibase + u][r], xv, acc[u]);
    }
  }
  const int j = nc0 + lane_j;
  if (j < n) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = kc0 + ibase + u;
      if (i < l) partial[((int64_t)g * n + j) * l + i] = acc[u];
    }
  }
}

void tile_range(int64_t m, int64_t row_offset, int64_t *tile0, int64_t *ntiles) {
  const int64_t t0 = row_offset / kTileRows;
  const int64_t t1 = (row_offset + m + kTileRows - 1) / kTileRows;
  *tile0 = t0;
  *ntiles = t1 - t0;
}

int choose_groups(int64_t ntiles, int64_t chunks) {
  const int64_t target = 4LL * num_sms();
  int64_t g = std::max<int64_t>(1, target / std::max<int64_t>(1, chunks));
  g = std::min<int64_t>(g, std::max<int64_t>(1, ntiles));
  return (int)std::min<int64_t>(g, 65535);
}

int colnorm_groups(int64_t m) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(2LL * num_sms(), (m + 4095) / 4096));
}

}  // namespace

int sketch_groups(int64_t m, int64_t n, int64_t k, int64_t row_offset) {
  int64_t tile0, ntiles;
  tile_range(m, row_offset, &tile0, &ntiles);
  const int64_t chunks = ((k + kChunkK - 1) / kChunkK) * ((n + kChunkN - 1) / kChunkN);
  return choose_groups(ntiles, chunks);
}

size_t sketch_workspace(int64_t m, int64_t n, int64_t k, int64_t row_offset, int prec) {
  Workspace w(nullptr, 0);
  w.take<char>(sketch_tc_workspace(m, n, k, row_offset, prec));
  return w.used;
}

// The sketch of the factorization path: the exact tensor-core kernel
// (sketch_tc.cu), whose exponent pre-pass also yields the column norms of the
// rank-revealing variant.
cudaError_t launch_sketch(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, int64_t k,
                          uint64_t seed, uint32_t stream_id, int64_t row_offset, double *P,
                          int64_t ldp, double *colnorm2, Workspace &ws, cudaStream_t st,
                          int *dev_status, int dist) {
  return launch_sketch_tc(X, m, n, ldx, prec, k, seed, stream_id, row_offset, P, ldp, colnorm2, dev_status, ws,
                          st, dist);
}

cudaError_t launch_sketch_into(const void *X, int64_t m, int64_t n, int64_t ldx, int prec,
                               int64_t k, uint64_t seed, int64_t row_offset, double *P,
                               int64_t ldp, double *colnorm2, double *scratch,
                               size_t scratch_doubles, cudaStream_t st) {
  int64_t tile0, ntiles;
  tile_range(m, row_offset, &tile0, &ntiles);
  const int64_t chunks = ((k + kChunkK - 1) / kChunkK) * ((n + kChunkN - 1) / kChunkN);
  int64_t groups = choose_groups(ntiles, chunks);
  const int cg = colnorm2 ? colnorm_groups(m) : 0;
  const int64_t room = (int64_t)scratch_doubles - (int64_t)cg * n;
  groups = std::min<int64_t>(groups, room / (n * k));
  if (groups < 1) return cudaErrorInvalidValue;
  double *partial = scratch;
  double *cp = scratch + groups * n * k;
  dim3 grid((unsigned)chunks, (unsigned)groups);
  const ThetaTable &tab = theta_table();
  switch (prec) {
    case RCQR_F64:
      sketch_partial_kernel<double><<<grid, kThreads, 0, st>>>(
          (const double *)X, m, (int)n, ldx, (int)k, seed, 0, row_offset, tile0, ntiles,
          (int)groups, tab, partial);
      break;
    case RCQR_F32:
      sketch_partial_kernel<float><<<grid, kThreads, 0, st>>>(
          (const float *)X, m, (int)n, ldx, (int)k, seed, 0, row_offset, tile0, ntiles,
          (int)groups, tab, partial);
      break;
    default:
      sketch_partial_kernel<__nv_bfloat16><<<grid, kThreads, 0, st>>>(
          (const __nv_bfloat16 *)X, m, (int)n, ldx, (int)k, seed, 0, row_offset, tile0, ntiles,
          (int)groups, tab, partial);
  }
  sketch_reduce_kernel<<<(unsigned)((k * n + 255) / 256), 256, 0, st>>>(
      partial, (int)groups, (int)k, (int)n, theta_scale(k), P, ldp);
  if (colnorm2) {
    switch (prec) {
      case RCQR_F64:
        colnorm_partial_kernel<double><<<cg, 256, 0, st>>>((const double *)X, m, (int)n, ldx, cg, cp);
        break;
      case RCQR_F32:
        colnorm_partial_kernel<float><<<cg, 256, 0, st>>>((const float *)X, m, (int)n, ldx, cg, cp);
        break;
      default:
        colnorm_partial_kernel<__nv_bfloat16><<<cg, 256, 0, st>>>((const __nv_bfloat16 *)X, m,
                                                                  (int)n, ldx, cg, cp);
    }
    colnorm_reduce_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(cp, cg, (int)n, colnorm2);
  }
  return cudaGetLastError();
}

size_t dense_left_workspace(int64_t l, int64_t m, int64_t n) {
  const int64_t chunks = ((l + kChunkK - 1) / kChunkK) * ((n + kChunkN - 1) / kChunkN);
  const int groups = choose_groups((m + kLRows - 1) / kLRows, chunks);
  Workspace w(nullptr, 0);
  w.take<double>((size_t)groups * n * l);
  return w.used;
}

cudaError_t launch_dense_left(const double *L, int64_t l, int64_t ldl, const void *X, int64_t m,
                              int64_t n, int64_t ldx, int prec, double *Y, int64_t ldy,
                              Workspace &ws, cudaStream_t st) {
  const int64_t chunks = ((l + kChunkK - 1) / kChunkK) * ((n + kChunkN - 1) / kChunkN);
  const int groups = choose_groups((m + kLRows - 1) / kLRows, chunks);
  double *partial = ws.take<double>((size_t)groups * n * l);
  if (!partial) return cudaErrorMemoryAllocation;
  dim3 grid((unsigned)chunks, (unsigned)groups);
  switch (prec) {
    case RCQR_F64:
      dense_left_partial_kernel<double><<<grid, kThreads, 0, st>>>(L, (int)l, ldl, (const double *)X,
                                                                  m, (int)n, ldx, groups, partial);
      break;
    case RCQR_F32:
      dense_left_partial_kernel<float><<<grid, kThreads, 0, st>>>(L, (int)l, ldl, (const float *)X,
                                                                 m, (int)n, ldx, groups, partial);
      break;
    default:
      dense_left_partial_kernel<__nv_bfloat16><<<grid, kThreads, 0, st>>>(
          L, (int)l, ldl, (const __nv_bfloat16 *)X, m, (int)n, ldx, groups, partial);
  }
  const int64_t total = l * n;
  sketch_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(partial, groups, (int)l,
                                                                        (int)n, 1.0, Y, ldy);
  return cudaGetLastError();
}

}  // namespace rcqr
