// Small dense FP64 kernels of the method (the matrices are at most 2048 x 256):
//  * Householder QR of the sketch P (Alg. 2 step 2; the paper's choice of
//    reflections, Sec. 3.1), diag(R) >= 0, S formed explicitly when asked;
//  * R alone by a tree over several CTAs (TSQR: leaf Householder QRs, then
//    folds of stacked triangles);
//  * column-pivoted Householder QR of P D^{-1}, the truncation rank and the
//    de-normalisation R <- R Pi^T D Pi (Alg. 7 steps 2, 3, 5 and Sec. 4);
//  * Cholesky of the Gram matrix with R <- R' R (Alg. 3 step 3);
//  * the inverse of an upper triangular matrix.
//
// GB300 issues FP64 at a few flops per clock per SM, so these kernels keep the
// FP64 instruction count minimal: one thread owns one column's dot product and
// update (no per-column shuffle reductions), the scalars of a reflector or a
// pivot are computed once and broadcast through shared memory, and the working
// copy has an odd leading dimension so that column-per-lane access is
// conflict-free.  The working copy lives in shared memory when it fits, else in
// the caller's workspace (L2 resident).
#include <algorithm>

#include "common.cuh"
#include "rcqr_internal.h"

namespace rcqr {

namespace {

constexpr int kSmallThreads = 256;
constexpr size_t kSmemLimit = 200 * 1024;
constexpr size_t kBatchedSmem = kSmemLimit;   // one batched QRCP CTA per SM (<= 128 per launch)

__device__ __forceinline__ int odd_ld(int rows) { return rows | 1; }

// Sum over lane-strided terms of warp 0 (call from warp 0 only): lane 0 gets the total.
__device__ __forceinline__ double warp0_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Dot products for the column updates: four threads per column, each summing
// every fourth row with four accumulators, the quarter sums combined by two
// shuffles (fixed order).  Returns the full sum in all four threads.
__device__ __forceinline__ double quad_dot(const double *a, const double *b, int i0, int i1, int q) {
  // four accumulators: FP64 latency, not throughput, bounds these short sums
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int i = i0 + q;
  for (; i + 12 < i1; i += 16) {
    s0 = fma(a[i], b[i], s0);
    s1 = fma(a[i + 4], b[i + 4], s1);
    s2 = fma(a[i + 8], b[i + 8], s2);
    s3 = fma(a[i + 12], b[i + 12], s3);
  }
  for (; i < i1; i += 4) s0 = fma(a[i], b[i], s0);
  double s = (s0 + s1) + (s2 + s3);
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  return s;
}

// One Householder step on column j of the rows x n matrix A (column-major, lda):
// v is built in A[j:, j] (A[j, j] <- v0); s_beta[j], s_diag[j] receive beta and
// the new diagonal entry; columns j+1.. are updated, one thread per column.
__device__ void householder_step(double *A, int rows, int n, int lda, int j, double *s_beta,
                                 double *s_diag) {
  double *col = A + (int64_t)j * lda;
  if (threadIdx.x < 32) {
    double t = 0.0, t1 = 0.0;
    int i = j + 1 + threadIdx.x;
    for (; i + 32 < rows; i += 64) {
      t = fma(col[i], col[i], t);
      t1 = fma(col[i + 32], col[i + 32], t1);
    }
    if (i < rows) t = fma(col[i], col[i], t);
    t = warp0_sum(t + t1);
    if (threadIdx.x == 0) {
      const double x0 = col[j];
      const double sigma = fma(x0, x0, t);
      double beta = 0.0, d = 0.0;
      if (sigma > 0.0) {
        const double alpha = sqrt(sigma);
        const double s = x0 >= 0.0 ? 1.0 : -1.0;
        const double v0 = x0 + s * alpha;
        beta = 2.0 / fma(v0, v0, t);
        d = -s * alpha;
        col[j] = v0;
      }
      s_beta[j] = beta;
      s_diag[j] = d;
    }
  }
  __syncthreads();
  const double beta = s_beta[j];
  if (beta != 0.0) {
    const int q = threadIdx.x & 3, nq = blockDim.x >> 2;
    // every warp runs the same iterations (the quad shuffles need all 32 lanes)
    for (int c0 = j + 1; c0 < n; c0 += nq) {
      const int c = c0 + (threadIdx.x >> 2);
      const bool valid = c < n;
      double *ac = A + (int64_t)(valid ? c : j) * lda;
      const double w = quad_dot(col, ac, j, valid ? rows : j, q);
      if (valid) {
        const double bw = beta * w;
        for (int i = j + q; i < rows; i += 4) ac[i] = fma(-bw, col[i], ac[i]);
      }
    }
  }
  __syncthreads();
}

// S = H_0 ... H_{n-1} [I; 0] from the reflectors stored in A (v in A[j:, j]).
__device__ void form_S(const double *A, int rows, int n, int lda, const double *s_beta, double *S,
                       int64_t lds) {
  for (int e = threadIdx.x; e < rows * n; e += blockDim.x) {
    const int i = e % rows, c = e / rows;
    S[i + (int64_t)c * lds] = (i == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = n - 1; j >= 0; --j) {
    const double beta = s_beta[j];
    if (beta != 0.0) {
      const double *v = A + (int64_t)j * lda;
      for (int c = j + threadIdx.x; c < n; c += blockDim.x) {
        double *sc = S + (int64_t)c * lds;
        double w = 0.0;
        for (int i = j; i < rows; ++i) w = fma(v[i], sc[i], w);
        const double bw = beta * w;
        for (int i = j; i < rows; ++i) sc[i] = fma(-bw, v[i], sc[i]);
      }
    }
    __syncthreads();
  }
}

// Copy rows r0..r0+rows-1 of P (ldp) into A (lda), optionally dividing column c by D[c].
__device__ void load_block(const double *P, int64_t ldp, int r0, int rows, int n, double *A, int lda,
                           const double *Dc) {
  for (int64_t e = threadIdx.x; e < (int64_t)rows * n; e += blockDim.x) {
    const int i = (int)(e % rows), c = (int)(e / rows);
    double v = P[(r0 + i) + (int64_t)c * ldp];
    if (Dc) v /= Dc[c];
    A[i + (int64_t)c * lda] = v;
  }
  __syncthreads();
}

// R (diag >= 0) from the Householder factors: row i negated when s_diag[i] < 0.
__device__ void store_R(const double *A, int lda, int n, const double *s_diag, double *R, int64_t ldr) {
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, c = e / n;
    const double sg = s_diag[i] < 0.0 ? -1.0 : 1.0;
    double v = 0.0;
    if (i < c) v = sg * A[i + (int64_t)c * lda];
    else if (i == c) v = sg * s_diag[i];
    R[i + (int64_t)c * ldr] = v;
  }
}

__global__ void __launch_bounds__(kSmallThreads)
small_qr_kernel(const double *__restrict__ P, int k, int n, int64_t ldp, double *S, int64_t lds,
                double *R, int64_t ldr, double *gwork, int use_smem) {
  extern __shared__ double smem[];
  __shared__ double s_beta[256], s_diag[256];
  double *A = use_smem ? smem : gwork;
  const int lda = odd_ld(k);
  load_block(P, ldp, 0, k, n, A, lda, nullptr);
  for (int j = 0; j < n; ++j) householder_step(A, k, n, lda, j, s_beta, s_diag);
  store_R(A, lda, n, s_diag, R, ldr);
  if (S) {
    form_S(A, k, n, lda, s_beta, S, lds);
    for (int e = threadIdx.x; e < k * n; e += blockDim.x) {
      const int i = e % k, c = e / k;
      if (s_diag[c] < 0.0) S[i + (int64_t)c * lds] = -S[i + (int64_t)c * lds];
    }
  }
}

// ---- R only, as a tree (TSQR): Householder QR of L row blocks of P on L CTAs,
// then the L triangles folded by one CTA.  R is unique once its diagonal is
// made positive, so it equals the R of Householder on all of P up to rounding.
__global__ void __launch_bounds__(kSmallThreads)
tsqr_leaf_kernel(const double *__restrict__ P, int k, int n, int64_t ldp, int L, double *Rleaf,
                 double *gwork, int use_smem) {
  extern __shared__ double smem[];
  __shared__ double s_beta[256], s_diag[256];
  const int l = blockIdx.x;
  const int r0 = (int)((int64_t)k * l / L), r1 = (int)((int64_t)k * (l + 1) / L);
  const int rows = r1 - r0;                       // >= n
  const int lda = odd_ld(rows);
  const int64_t per = (int64_t)odd_ld((k + L - 1) / L) * n;
  double *A = use_smem ? smem : gwork + (int64_t)l * per;
  load_block(P, ldp, r0, rows, n, A, lda, nullptr);
  for (int j = 0; j < n; ++j) householder_step(A, rows, n, lda, j, s_beta, s_diag);
  double *Rl = Rleaf + (int64_t)l * n * n;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, c = e / n;
    Rl[e] = i < c ? A[i + (int64_t)c * lda] : (i == c ? s_diag[i] : 0.0);
  }
}

// T <- R of [T; B] for upper triangular n x n T and B (column-major, leading
// dimension ld).  The reflector of column j acts on row j of T and rows 0..j of B only.
__device__ void fold_triangles(double *T, double *B, int n, int ld, double *scal) {
  for (int j = 0; j < n; ++j) {
    double *bj = B + (int64_t)j * ld;
    if (threadIdx.x < 32) {
      double t = 0.0;
      for (int i = threadIdx.x; i <= j; i += 32) t = fma(bj[i], bj[i], t);
      t = warp0_sum(t);
      if (threadIdx.x == 0) {
        const double x0 = T[j + (int64_t)j * ld];
        double beta = 0.0, v0 = 0.0, d = x0;
        if (t > 0.0) {
          const double alpha = sqrt(fma(x0, x0, t));
          const double s = x0 >= 0.0 ? 1.0 : -1.0;
          v0 = x0 + s * alpha;
          beta = 2.0 / fma(v0, v0, t);
          d = -s * alpha;
        }
        scal[0] = v0;
        scal[1] = beta;
        scal[2] = d;
      }
    }
    __syncthreads();
    const double v0 = scal[0], beta = scal[1];
    if (beta != 0.0) {
      const int q = threadIdx.x & 3, nq = blockDim.x >> 2;
      for (int c0 = j + 1; c0 < n; c0 += nq) {
        const int c = c0 + (threadIdx.x >> 2);
        const bool valid = c < n;
        double *bc = B + (int64_t)(valid ? c : j) * ld;
        const double tjc = valid ? T[j + (int64_t)c * ld] : 0.0;
        const double w = fma(v0, tjc, quad_dot(bj, bc, 0, valid ? j + 1 : 0, q));
        if (valid) {
          const double bw = beta * w;
          for (int i = q; i <= j; i += 4) bc[i] = fma(-bw, bj[i], bc[i]);
          if (q == 0) T[j + (int64_t)c * ld] = fma(-bw, v0, tjc);
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) T[j + (int64_t)j * ld] = scal[2];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) bj[i] = 0.0;
    __syncthreads();
  }
}

// Folds the L leaf triangles into one.  The triangles are staged in shared
// memory (odd leading dimension, conflict-free column-per-quad access) when
// they fit, so the n sequential steps of each fold run on shared memory rather
// than L2; otherwise they are folded in place in the workspace.
__global__ void __launch_bounds__(kSmallThreads)
tsqr_fold_kernel(double *Rleaf, int n, int L, double *R, int64_t ldr, int use_smem) {
  extern __shared__ double smem[];
  __shared__ double scal[4];
  const int ld = use_smem ? (n | 1) : n;
  double *W = use_smem ? smem : Rleaf;
  if (use_smem) {
    for (int64_t e = threadIdx.x; e < (int64_t)L * n * n; e += blockDim.x) {
      const int l = (int)(e / ((int64_t)n * n)), rem = (int)(e % ((int64_t)n * n));
      const int i = rem % n, c = rem / n;
      W[(int64_t)l * n * ld + i + (int64_t)c * ld] = Rleaf[e];
    }
    __syncthreads();
  }
  for (int l = 1; l < L; ++l) fold_triangles(W, W + (int64_t)l * n * ld, n, ld, scal);
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, c = e / n;
    const double sg = W[i + (int64_t)i * ld] < 0.0 ? -1.0 : 1.0;
    R[i + (int64_t)c * ldr] = i <= c ? sg * W[i + (int64_t)c * ld] : 0.0;
  }
}

// One level of the fold tree: CTA b folds leaf triangle (2b + 1) stride into
// leaf 2b stride (in place in the workspace).
__global__ void __launch_bounds__(kSmallThreads)
tsqr_pair_kernel(double *Rleaf, int n, int L, int stride) {
  __shared__ double scal[4];
  const int64_t t = (int64_t)2 * blockIdx.x * stride, u = t + stride;
  if (u >= L) return;
  fold_triangles(Rleaf + t * n * n, Rleaf + u * n * n, n, n, scal);
}

// ---- R only on a cluster of 8 CTAs (k <= 32 RPL rows, n <= 64 CPW columns).
// Householder QR distributed by columns: column g lives in the registers of one
// warp (CTA g % 8, warp (g / 8) % 8, slot g / 64), lane l holding rows l, l + 32,
// ...  Step j: every warp applies reflector j (read from its own shared memory)
// to its columns > j; the warp that owns column j + 1 then forms reflector
// j + 1 and stores it into the shared memory of all eight CTAs (distributed
// shared memory), and one cluster barrier publishes it.  The reflector buffers
// alternate between two slots, so one barrier per column suffices: a slot is
// rewritten only after every CTA has passed the barrier that followed its
// last read.  The trailing updates of a step run on eight SMs at once and the
// chain of dependent operations per column (dot, update, norm, square root) is
// one warp's.  Same reflections and the same diag(R) >= 0 convention as the
// one-CTA kernels.
constexpr int kClusterQR = 8;

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t map_shared(const void *p, uint32_t rank) {
  uint32_t local = static_cast<uint32_t>(__cvta_generic_to_shared(p)), remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
  return remote;
}

__device__ __forceinline__ void st_cluster_f64(uint32_t addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}

__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

__device__ __forceinline__ double warp_allsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int RPL, int CPW>
__global__ void __cluster_dims__(kClusterQR, 1, 1) __launch_bounds__(kSmallThreads)
cluster_r_kernel(const double *__restrict__ P, int k, int n, int64_t ldp, double *R, int64_t ldr) {
  __shared__ double vbuf[2][32 * RPL];
  __shared__ double s_beta[64 * CPW], s_diag[64 * CPW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t crank = cluster_rank();
  double a[CPW][RPL];
  int g[CPW];
#pragma unroll
  for (int s = 0; s < CPW; ++s) {
    g[s] = (int)crank + kClusterQR * (warp + 8 * s);
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int row = lane + 32 * t;
      a[s][t] = (g[s] < n && row < k) ? P[row + (int64_t)g[s] * ldp] : 0.0;
    }
  }
  uint32_t rv[kClusterQR];
#pragma unroll
  for (int c = 0; c < kClusterQR; ++c) rv[c] = map_shared(&vbuf[0][0], c);
  // Reflector of column jj from slot s's registers: v = [0 .. 0, v0, a(jj+1:)],
  // beta = 2 / v^T v, diag = -sign(x0) ||a(jj:)||; stored into every CTA's slot jj & 1.
  auto reflect = [&](int s, int jj) {
    double t = 0.0, x0 = 0.0;
#pragma unroll
    for (int u = 0; u < RPL; ++u) {
      const int row = lane + 32 * u;
      if (row > jj) t = fma(a[s][u], a[s][u], t);
      if (row == jj) x0 = a[s][u];
    }
    t = warp_allsum(t);
    x0 = __shfl_sync(0xffffffffu, x0, jj & 31);
    double beta = 0.0, d = 0.0, v0 = x0;
    const double sigma = fma(x0, x0, t);
    if (sigma > 0.0) {
      const double alpha = sqrt(sigma);
      const double sg = x0 >= 0.0 ? 1.0 : -1.0;
      v0 = x0 + sg * alpha;
      beta = 2.0 / fma(v0, v0, t);
      d = -sg * alpha;
    }
    const uint32_t off = (uint32_t)((jj & 1) * 32 * RPL) * 8u;
#pragma unroll
    for (int u = 0; u < RPL; ++u) {
      const int row = lane + 32 * u;
      const double v = row < jj ? 0.0 : (row == jj ? v0 : a[s][u]);
#pragma unroll
      for (int c = 0; c < kClusterQR; ++c) st_cluster_f64(rv[c] + off + (uint32_t)row * 8u, v);
    }
    if (lane < kClusterQR) {
      st_cluster_f64(map_shared(&s_beta[jj], lane), beta);
      st_cluster_f64(map_shared(&s_diag[jj], lane), d);
    }
  };
  cluster_barrier();   // every CTA of the cluster is running before the first remote store
  if (crank == 0 && warp == 0) reflect(0, 0);
  cluster_barrier();
  for (int j = 0; j < n; ++j) {
    const double *v = vbuf[j & 1];
    const double beta = s_beta[j];
#pragma unroll
    for (int s = 0; s < CPW; ++s) {
      if (g[s] > j && g[s] < n) {   // warp-uniform
        if (beta != 0.0) {
          double w = 0.0;
#pragma unroll
          for (int u = 0; u < RPL; ++u) w = fma(v[lane + 32 * u], a[s][u], w);
          const double bw = beta * warp_allsum(w);
#pragma unroll
          for (int u = 0; u < RPL; ++u) a[s][u] = fma(-bw, v[lane + 32 * u], a[s][u]);
        }
        if (g[s] == j + 1) reflect(s, j + 1);
      }
    }
    cluster_barrier();
  }
  // R = diag(sign d) * (upper triangle; diagonal d)
#pragma unroll
  for (int s = 0; s < CPW; ++s) {
    if (g[s] < n) {
#pragma unroll
      for (int u = 0; u < RPL; ++u) {
        const int row = lane + 32 * u;
        if (row < n) {
          const double sg = s_diag[row < g[s] ? row : g[s]] < 0.0 ? -1.0 : 1.0;
          double val = 0.0;
          if (row < g[s]) val = sg * a[s][u];
          else if (row == g[s]) val = sg * s_diag[row];
          R[row + (int64_t)g[s] * ldr] = val;
        }
      }
    }
  }
}

// Copy P[:, perm] D^{-1} (columns permuted and normalised) into A (lda).
__device__ void load_permuted(const double *P, int64_t ldp, int k, int n, const int *perm, const double *Dc,
                              double *A, int lda) {
  for (int64_t e = threadIdx.x; e < (int64_t)k * n; e += blockDim.x) {
    const int i = (int)(e % k), c = (int)(e / k);
    const int src = perm[c];
    A[i + (int64_t)c * lda] = P[i + (int64_t)src * ldp] / Dc[src];
  }
  __syncthreads();
}

// ||R||_2 (R n x n upper) by power iteration on R^T R from the all-ones vector, until the
// estimate ||R x|| / ||x|| (non-decreasing) grows by at most 1e-13 of itself, at most 100
// steps.  Every thread returns the estimate.
__device__ double spectral_norm_est(const double *R, int64_t ldr, int n, double *s_x, double *s_y, double *s_t,
                                    double *s_scal) {
  for (int c = threadIdx.x; c < n; c += blockDim.x) s_x[c] = 1.0;
  __syncthreads();
  double norm2 = 0.0;
  for (int it = 0; it < 100; ++it) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {  // y = R x
      double sacc = 0.0;
      for (int c = i; c < n; ++c) sacc = fma(R[i + (int64_t)c * ldr], s_x[c], sacc);
      s_y[i] = sacc;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      double yy = 0.0, xx = 0.0;
      for (int c = threadIdx.x; c < n; c += 32) {
        yy = fma(s_y[c], s_y[c], yy);
        xx = fma(s_x[c], s_x[c], xx);
      }
      yy = warp0_sum(yy);
      xx = warp0_sum(xx);
      if (threadIdx.x == 0) s_scal[0] = xx > 0.0 ? sqrt(yy / xx) : 0.0;   // ||R x|| / ||x||
    }
    for (int c = threadIdx.x; c < n; c += blockDim.x) {  // x' = R^T y
      double sacc = 0.0;
      for (int i = 0; i <= c; ++i) sacc = fma(R[i + (int64_t)c * ldr], s_y[i], sacc);
      s_t[c] = sacc;
    }
    __syncthreads();
    const double est = s_scal[0];
    const bool done = it >= 2 && est - norm2 <= 1e-13 * est;
    norm2 = est;
    if (threadIdx.x < 32) {
      double nn = 0.0;
      for (int c = threadIdx.x; c < n; c += 32) nn = fma(s_t[c], s_t[c], nn);
      nn = warp0_sum(nn);
      if (threadIdx.x == 0) s_scal[1] = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) s_x[c] = s_t[c] * s_scal[1];
    __syncthreads();
    if (done) break;
  }
  return norm2;
}

// Alg. 7 step 3: the least r with ||R[r:, r:]||_F <= tau ||R||_2 (thread 0; returned to all).
__device__ int truncation_rank_dev(const double *R, int64_t ldr, int n, double tau, double norm2, double *s_y,
                                   int *s_out) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double sacc = 0.0;
    for (int c = i; c < n; ++c) sacc = fma(R[i + (int64_t)c * ldr], R[i + (int64_t)c * ldr], sacc);
    s_y[i] = sacc;    // row i's share of the suffix Frobenius norms
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double bound = tau * norm2;
    double suffix = 0.0;
    int r = n;
    // F2[r] = sum_{i >= r} s_y[i] is non-increasing in r
    for (int rr = n; rr >= 0; --rr) {
      if (rr < n) suffix += s_y[rr];
      if (sqrt(suffix) <= bound) r = rr;
      else break;
    }
    *s_out = r;
  }
  __syncthreads();
  return *s_out;
}

// Strong-RRQR swaps (Gu & Eisenstat 1996, Algorithm 4) at rank r on the normalised R of
// P[:, perm] D^{-1}: while the largest
//   rho_ij = (R11^{-1} R12)_ij^2 + (gamma_j(R22) / omega_i(R11))^2
// (gamma_j: 2-norm of column j of R22, omega_i: 1 / 2-norm of row i of R11^{-1}; the first
// maximum in column-major order on ties) exceeds f^2, columns i and r + j trade places and
// P[:, perm] D^{-1} is factored again by Householder QR.  sqrt(rho_ij) is the growth of
// |det R11| under that swap, so the loop ends; at most 4 n swaps.  W (r n doubles of scratch)
// holds R11^{-1} (r x r) and R11^{-1} R12 (r x (n - r)), both with leading dimension r.
__device__ void strong_swaps(const double *P, int k, int n, int64_t ldp, double *R, int64_t ldr, double *A, int lda,
                             double *W, int r, double f, int *s_perm, const double *s_D, double *s_w, double *s_g,
                             double *s_beta, double *s_diag, unsigned long long *s_bkey, int *s_bidx) {
  if (r <= 0 || r >= n) return;
  const int nr = n - r;
  double *Wi = W, *W12 = W + (int64_t)r * r;
  for (int sw = 0; sw < 4 * n; ++sw) {
    // columns of R11^{-1} and of R11^{-1} R12 by back substitution, one thread per column
    for (int c = threadIdx.x; c < r + nr; c += blockDim.x) {
      double *out = c < r ? Wi + (int64_t)c * r : W12 + (int64_t)(c - r) * r;
      const int top = c < r ? c : r - 1;
      for (int i = r - 1; i > top; --i) out[i] = 0.0;
      for (int i = top; i >= 0; --i) {
        double x = c < r ? (i == c ? 1.0 : 0.0) : R[i + (int64_t)c * ldr];
        for (int t = i + 1; t <= top; ++t) x = fma(-R[i + (int64_t)t * ldr], out[t], x);
        out[i] = x / R[i + (int64_t)i * ldr];
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < r; i += blockDim.x) {     // 1 / omega_i^2
      double sacc = 0.0;
      for (int c = i; c < r; ++c) sacc = fma(Wi[i + (int64_t)c * r], Wi[i + (int64_t)c * r], sacc);
      s_w[i] = sacc;
    }
    for (int j = threadIdx.x; j < nr; j += blockDim.x) {    // gamma_j^2
      double sacc = 0.0;
      for (int t = r; t <= r + j; ++t) sacc = fma(R[t + (int64_t)(r + j) * ldr], R[t + (int64_t)(r + j) * ldr], sacc);
      s_g[j] = sacc;
    }
    __syncthreads();
    unsigned long long best = 0;
    int bidx = -1;
    for (int t = threadIdx.x; t < r * nr; t += blockDim.x) {
      const int i = t % r, j = t / r;
      const double w = W12[i + (int64_t)j * r];
      const double rho = fma(w, w, s_w[i] * s_g[j]);
      const unsigned long long key = rho >= 0.0 ? (unsigned long long)__double_as_longlong(rho) : 0ull;
      if (bidx < 0 || key > best) {    // t increases: on a tie the first (lowest) t stays
        best = key;
        bidx = t;
      }
    }
    s_bkey[threadIdx.x] = best;
    s_bidx[threadIdx.x] = bidx;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long bk = 0;
      int bt = -1;
      for (int u = 0; u < (int)blockDim.x; ++u) {
        const int t = s_bidx[u];
        if (t < 0) continue;
        if (bt < 0 || s_bkey[u] > bk || (s_bkey[u] == bk && t < bt)) {
          bk = s_bkey[u];
          bt = t;
        }
      }
      const double rho = __longlong_as_double((long long)bk);
      s_bidx[0] = (bt >= 0 && rho > f * f) ? bt : -1;
      if (s_bidx[0] >= 0) {
        const int i = bt % r, j = bt / r;
        const int tmp = s_perm[i];
        s_perm[i] = s_perm[r + j];
        s_perm[r + j] = tmp;
      }
    }
    __syncthreads();
    if (s_bidx[0] < 0) break;
    __syncthreads();
    load_permuted(P, ldp, k, n, s_perm, s_D, A, lda);
    for (int j = 0; j < n; ++j) householder_step(A, k, n, lda, j, s_beta, s_diag);
    store_R(A, lda, n, s_diag, R, ldr);
    __syncthreads();
  }
}

// Column-pivoted QR of P D^{-1} + rank + de-normalised R; f > 0: followed by the
// strong-RRQR swaps at the truncation rank (repeated while the rank of the swapped factor
// changes, at most 4 rounds).
__device__ void qrcp_body(const double *__restrict__ P, int k, int n, int64_t ldp, const double *colnorm2,
                          double tau, double f, double *R, int64_t ldr, int32_t *perm_out, int64_t *rank_out,
                          int *dev_status, double *gwork, int use_smem, double *wscratch) {
  extern __shared__ double smem[];
  __shared__ double s_beta[256], s_diag[256], s_D[256], s_x[256], s_y[256], s_scal[4];
  __shared__ unsigned long long s_key[256];
  __shared__ int s_perm[256], s_bidx[256];
  __shared__ int s_piv;
  double *A = use_smem ? smem : gwork;
  const int lda = odd_ld(k);
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    const double d = colnorm2 ? sqrt(colnorm2[c]) : 1.0;
    s_D[c] = d > 0.0 ? d : 1.0;
    s_perm[c] = c;
  }
  __syncthreads();
  load_block(P, ldp, 0, k, n, A, lda, s_D);
  for (int j = 0; j < n; ++j) {
    // recomputed norms of the remaining columns (rows j..k-1), one thread per column;
    // non-negative doubles order like their bit patterns
    for (int c = j + threadIdx.x; c < n; c += blockDim.x) {
      const double *ac = A + (int64_t)c * lda;
      double sacc = 0.0;
      for (int i = j; i < k; ++i) sacc = fma(ac[i], ac[i], sacc);
      s_key[c] = (unsigned long long)__double_as_longlong(sqrt(sacc));
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      // argmax, lowest index on ties
      unsigned long long best = 0;
      int p = n;
      for (int c = j + threadIdx.x; c < n; c += 32) {
        const unsigned long long kv = s_key[c];
        if (p == n || kv > best) {
          best = kv;
          p = c;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_down_sync(0xffffffffu, best, o);
        const int op = __shfl_down_sync(0xffffffffu, p, o);
        if (op < n && (p == n || ob > best || (ob == best && op < p))) {
          best = ob;
          p = op;
        }
      }
      if (threadIdx.x == 0) s_piv = p;
    }
    __syncthreads();
    const int p = s_piv;
    if (p != j) {
      for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const double a = A[i + (int64_t)j * lda];
        A[i + (int64_t)j * lda] = A[i + (int64_t)p * lda];
        A[i + (int64_t)p * lda] = a;
      }
      if (threadIdx.x == 0) {
        const int t = s_perm[j];
        s_perm[j] = s_perm[p];
        s_perm[p] = t;
      }
    }
    __syncthreads();
    householder_step(A, k, n, lda, j, s_beta, s_diag);
  }
  store_R(A, lda, n, s_diag, R, ldr);
  __syncthreads();
  double norm2 = spectral_norm_est(R, ldr, n, s_x, s_y, s_beta, s_scal);
  int r = truncation_rank_dev(R, ldr, n, tau, norm2, s_y, &s_piv);
  if (f > 0.0) {
    double *W = wscratch ? wscratch : A;       // A is reloaded after every swap decision
    for (int round = 0; round < 4 && r > 0 && r < n; ++round) {
      strong_swaps(P, k, n, ldp, R, ldr, A, lda, W, r, f, s_perm, s_D, s_x, s_y, s_beta, s_diag, s_key, s_bidx);
      norm2 = spectral_norm_est(R, ldr, n, s_x, s_y, s_beta, s_scal);
      const int r2 = truncation_rank_dev(R, ldr, n, tau, norm2, s_y, &s_piv);
      if (r2 == r) break;
      r = r2;
    }
  }
  if (threadIdx.x == 0) {
    *rank_out = r;
    // the first error of a call is kept (an earlier one, e.g. a timed-out sketch, wins)
    if (r == 0 && dev_status && atomicCAS(dev_status, 0, (int)RCQR_ERANK0) == 0) dev_status[1] = -1;
  }
  for (int c = threadIdx.x; c < n; c += blockDim.x) perm_out[c] = s_perm[c];
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, c = e / n;
    const double v = R[i + (int64_t)c * ldr];
    R[i + (int64_t)c * ldr] = (i < r) ? v * s_D[s_perm[c]] : 0.0;
  }
}

__global__ void __launch_bounds__(kSmallThreads)
qrcp_kernel(const double *__restrict__ P, int k, int n, int64_t ldp, const double *colnorm2, double tau, double f,
            double *R, int64_t ldr, int32_t *perm_out, int64_t *rank_out, int *dev_status, double *gwork, int use_smem) {
  // the swap scratch shares gwork when the working copy lives in shared memory
  qrcp_body(P, k, n, ldp, colnorm2, tau, f, R, ldr, perm_out, rank_out, dev_status, gwork, use_smem,
            use_smem ? gwork : nullptr);
}

// Many QRCPs in one launch (a batch of factorizations): CTA b runs job b, with its
// working copy in shared memory when it fits the launch's allotment.
struct QrcpJobs {
  QrcpJob j[kQrcpJobsPerLaunch];
};

__global__ void __launch_bounds__(kSmallThreads)
qrcp_batched_kernel(const __grid_constant__ QrcpJobs jobs, double tau, double f, int64_t smem_doubles) {
  const QrcpJob &jb = jobs.j[blockIdx.x];
  const bool sm = (int64_t)odd_ld(jb.k) * jb.n <= smem_doubles;
  qrcp_body(jb.P, jb.k, jb.n, jb.ldp, jb.colnorm2, tau, f, jb.R, jb.ldr, jb.perm, jb.rank, jb.status, jb.gwork, sm,
            sm ? jb.gwork : nullptr);
}

// R' = chol(A[:r,:r]) (Alg. 3 step 3) on one CTA: left-looking on a shared-memory
// copy of R' (odd leading dimension) when it fits.  Step j forms, four threads
// per column, the dots of column j of R' with columns j..r-1 over rows 0..j-1;
// one thread takes the pivot's square root and reciprocal (GB300's FP64 unit
// runs a warp instruction in ~16 cycles, so redundant pivots in every thread
// cost more than the barrier that broadcasts one), and row j is finished by
// multiplication.  A failed pivot leaves R'_jj = 0, which the apply kernel
// checks.  (R' only; the update R <- R' R is chol_apply_kernel.)
constexpr size_t kCholSmem = 160 * 1024;

__global__ void __launch_bounds__(kSmallThreads)
chol_factor_kernel(const double *__restrict__ A, int n, int64_t lda, const int64_t *rank, double *Rp, int64_t ldrp,
                   int *dev_status, int use_smem) {
  extern __shared__ double smem[];
  __shared__ double s_dot[256];
  __shared__ double s_inv;
  __shared__ int s_fail;
  const int r = rank ? (int)(*rank < (int64_t)n ? *rank : (int64_t)n) : n;
  const int64_t ldw = use_smem ? (n | 1) : ldrp;
  double *W = use_smem ? smem : Rp;
  if (threadIdx.x == 0) s_fail = -1;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) W[(e % n) + (int64_t)(e / n) * ldw] = 0.0;
  __syncthreads();
  const int q = threadIdx.x & 3, nq = blockDim.x >> 2;
  for (int j = 0; j < r; ++j) {
    const double *cj = W + (int64_t)j * ldw;
    for (int c0 = j; c0 < r; c0 += nq) {
      const int c = c0 + (threadIdx.x >> 2);
      const bool valid = c < r;
      const double dot = quad_dot(cj, W + (int64_t)(valid ? c : j) * ldw, 0, valid ? j : 0, q);
      if (valid && q == 0) s_dot[c] = dot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const double d = A[j + (int64_t)j * lda] - s_dot[j];
      if (!(d > 0.0)) {
        s_fail = j;
      } else {
        const double djj = sqrt(d);
        W[j + (int64_t)j * ldw] = djj;
        s_inv = 1.0 / djj;
      }
    }
    __syncthreads();
    if (s_fail >= 0) break;
    const double inv = s_inv;
    for (int c = j + 1 + threadIdx.x; c < r; c += blockDim.x)
      W[j + (int64_t)c * ldw] = (A[j + (int64_t)c * lda] - s_dot[c]) * inv;
    __syncthreads();
  }
  if (s_fail >= 0) {
    // the first error of a call is kept (an earlier one, e.g. a timed-out sketch, wins)
    if (threadIdx.x == 0 && dev_status && atomicCAS(dev_status, 0, (int)RCQR_ENOTSPD) == 0) dev_status[1] = s_fail;
  }
  if (use_smem)
    for (int e = threadIdx.x; e < n * n; e += blockDim.x)
      Rp[(e % n) + (int64_t)(e / n) * ldrp] = W[(e % n) + (int64_t)(e / n) * ldw];
}

// R[:r, c] <- R' R[:r, c] (Alg. 3 step 3's update of the first pass's R), one
// CTA per column c: column c of the product depends only on column c of the
// old R, so the columns are updated in place independently.  For n <= 64 the
// block R'[0..c, 0..c] is staged in shared memory first, eight independent
// loads per thread in flight (not one L2 round trip per element).  Nothing is
// written if R' has a non-positive diagonal entry (a failed Cholesky).
constexpr int kApplyThreads = 64;

__global__ void __launch_bounds__(kApplyThreads)
chol_apply_kernel(const double *__restrict__ Rp, int n, int64_t ldrp, const int64_t *rank, double *R, int64_t ldr) {
  __shared__ double s_col[256];
  __shared__ double s_R[64 * 65];     // R'[0..ce, 0..ce] (column stride 65), n <= 64
  __shared__ int s_bad;
  const int c = blockIdx.x;
  const int r = rank ? (int)(*rank < (int64_t)n ? *rank : (int64_t)n) : n;
  const bool staged = n <= 64;
  const int ce = min(c, r - 1);       // last row / column of R' this column needs
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < r; i += blockDim.x)
    if (!(Rp[i + (int64_t)i * ldrp] > 0.0)) s_bad = 1;
  for (int i = threadIdx.x; i < r; i += blockDim.x) s_col[i] = R[i + (int64_t)c * ldr];
  if (staged && ce >= 0) {
    const int cnt = (ce + 1) * (ce + 1);
    for (int e0 = threadIdx.x; e0 < cnt; e0 += 8 * blockDim.x) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * blockDim.x;
        v[u] = e < cnt ? Rp[(e % (ce + 1)) + (int64_t)(e / (ce + 1)) * ldrp] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < cnt) s_R[(e % (ce + 1)) + (e / (ce + 1)) * 65] = v[u];
      }
    }
  }
  __syncthreads();
  if (s_bad) return;   // R untouched
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    double s = 0.0;
    if (staged)
      for (int l = i; l <= ce; ++l) s = fma(s_R[i + l * 65], s_col[l], s);
    else
      for (int l = i; l <= ce; ++l) s = fma(Rp[i + (int64_t)l * ldrp], s_col[l], s);
    R[i + (int64_t)c * ldr] = c >= i ? s : 0.0;
  }
}

// W = R^{-1} on the leading r x r block (zero elsewhere): column c by back substitution.
__global__ void tri_inverse_kernel(const double *__restrict__ R, int n, int64_t ldr,
                                   const int64_t *rank, double *W, int64_t ldw) {
  const int r = rank ? (int)(*rank < (int64_t)n ? *rank : (int64_t)n) : n;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    double *w = W + (int64_t)c * ldw;
    for (int i = 0; i < n; ++i) w[i] = 0.0;
    if (c >= r) continue;
    w[c] = 1.0 / R[c + (int64_t)c * ldr];
    for (int i = c - 1; i >= 0; --i) {
      double s = 0.0;
      for (int l = i + 1; l <= c; ++l) s = fma(R[i + (int64_t)l * ldr], w[l], s);
      w[i] = -s / R[i + (int64_t)i * ldr];
    }
  }
}

__global__ void reset_status_kernel(int *st) {
  st[0] = RCQR_OK;
  st[1] = -1;
}

__global__ void set_rank_kernel(int64_t *rank, int64_t v) { *rank = v; }

size_t copy_bytes(int64_t rows, int64_t n) { return (size_t)((rows | 1) * n) * 8; }
bool fits_smem(int64_t rows, int64_t n) { return copy_bytes(rows, n) <= kSmemLimit; }

// Leaves of the TSQR tree.  Every Householder step is a chain of dependent FP64
// operations (a reduction, a square root, a division) of a few microseconds on
// GB300, and a tree costs n steps per level, so small problems (n <= 64, k <= 4n)
// are factored by one CTA.  Larger ones are bound by FP64 throughput on that one
// SM (about k n^2 multiply-adds at ~2 per clock): square leaves spread that work,
// and the folds run as a binary tree, one level per launch.
int tsqr_leaves(int64_t k, int64_t n) {
  if (n <= 64 && k <= 4 * n) return 1;
  return (int)std::max<int64_t>(1, std::min<int64_t>(k / n, 32));
}

// The cluster kernel covers the sketches of up to 512 rows and 128 columns
// (k <= 4n there, the shapes whose one-CTA Householder is FP64-throughput bound).
bool cluster_r_supported(int64_t k, int64_t n) { return n <= 128 && k <= 512 && k >= n; }

}  // namespace

size_t small_qr_workspace(int64_t k, int64_t n) {
  const int L = tsqr_leaves(k, n);
  Workspace w(nullptr, 0);
  w.take<double>((size_t)((k + L) | 1) * n + (size_t)2 * L * n);   // working copies
  w.take<double>((size_t)L * n * n);                                // leaf triangles
  return w.used;
}

cudaError_t launch_small_r(const double *P, int64_t k, int64_t n, int64_t ldp, double *R, int64_t ldr,
                           Workspace &ws, cudaStream_t st) {
  if (cluster_r_supported(k, n)) {
    const int rpl = k <= 64 ? 2 : (k <= 128 ? 4 : (k <= 256 ? 8 : 16));
#define RCQR_CLUSTER_R(RP)                                                                           \
  case RP:                                                                                           \
    if (n <= 64)                                                                                     \
      cluster_r_kernel<RP, 1><<<kClusterQR, kSmallThreads, 0, st>>>(P, (int)k, (int)n, ldp, R, ldr); \
    else                                                                                             \
      cluster_r_kernel<RP, 2><<<kClusterQR, kSmallThreads, 0, st>>>(P, (int)k, (int)n, ldp, R, ldr); \
    break;
    switch (rpl) {
      RCQR_CLUSTER_R(2)
      RCQR_CLUSTER_R(4)
      RCQR_CLUSTER_R(8)
      RCQR_CLUSTER_R(16)
    }
#undef RCQR_CLUSTER_R
    return cudaGetLastError();
  }
  const int L = tsqr_leaves(k, n);
  double *g = ws.take<double>((size_t)((k + L) | 1) * n + (size_t)2 * L * n);
  double *Rleaf = ws.take<double>((size_t)L * n * n);
  if (!g || !Rleaf) return cudaErrorMemoryAllocation;
  const int64_t rows_max = (k + L - 1) / L;
  const bool sm = fits_smem(rows_max, n);
  const size_t bytes = sm ? copy_bytes(rows_max, n) : 0;
  if (sm) set_smem(tsqr_leaf_kernel, (int)kSmemLimit);
  tsqr_leaf_kernel<<<L, kSmallThreads, bytes, st>>>(P, (int)k, (int)n, ldp, L, Rleaf, g, sm);
  int Lf = L;   // leaves left for the final kernel
  const size_t fold_bytes = (size_t)L * n * (n | 1) * 8;
  if (L > 2 && fold_bytes > kSmemLimit) {
    // binary tree in the workspace; the final kernel sees one triangle
    for (int stride = 1; stride < L; stride *= 2)
      tsqr_pair_kernel<<<(unsigned)((L + 2 * stride - 1) / (2 * stride)), kSmallThreads, 0, st>>>(Rleaf, (int)n, L,
                                                                                                  stride);
    Lf = 1;
  }
  const size_t final_bytes = (size_t)Lf * n * (n | 1) * 8;
  const bool fold_sm = final_bytes <= kSmemLimit;
  if (fold_sm) set_smem(tsqr_fold_kernel, (int)kSmemLimit);
  tsqr_fold_kernel<<<1, kSmallThreads, fold_sm ? final_bytes : 0, st>>>(Rleaf, (int)n, Lf, R, ldr, fold_sm);
  return cudaGetLastError();
}

cudaError_t launch_small_qr(const double *P, int64_t k, int64_t n, int64_t ldp, double *S,
                            int64_t lds, double *R, int64_t ldr, Workspace &ws, cudaStream_t st) {
  const bool sm = fits_smem(k, n);
  double *g = ws.take<double>((size_t)(k | 1) * n);
  if (!g) return cudaErrorMemoryAllocation;
  const size_t bytes = sm ? copy_bytes(k, n) : 0;
  if (sm) set_smem(small_qr_kernel, (int)kSmemLimit);
  small_qr_kernel<<<1, kSmallThreads, bytes, st>>>(P, (int)k, (int)n, ldp, S, lds, R, ldr, g, sm);
  return cudaGetLastError();
}

cudaError_t launch_qrcp(const double *P, int64_t k, int64_t n, int64_t ldp, const double *colnorm2,
                        double tau, double *R, int64_t ldr, int32_t *perm, int64_t *rank,
                        int *dev_status, Workspace &ws, cudaStream_t st, double f) {
  const bool sm = fits_smem(k, n);
  double *g = ws.take<double>((size_t)(k | 1) * n);
  if (!g) return cudaErrorMemoryAllocation;
  const size_t bytes = sm ? copy_bytes(k, n) : 0;
  if (sm) set_smem(qrcp_kernel, (int)kSmemLimit);
  qrcp_kernel<<<1, kSmallThreads, bytes, st>>>(P, (int)k, (int)n, ldp, colnorm2, tau, f, R, ldr, perm,
                                               rank, dev_status, g, sm);
  return cudaGetLastError();
}

size_t qrcp_work_doubles(int64_t k, int64_t n) { return (size_t)(k | 1) * n; }

cudaError_t launch_qrcp_jobs(const QrcpJob *jobs, int count, double tau, cudaStream_t st, double f) {
  if (count < 1 || count > kQrcpJobsPerLaunch) return cudaErrorInvalidValue;
  QrcpJobs pj;
  int64_t need = 0;
  for (int b = 0; b < count; ++b) {
    pj.j[b] = jobs[b];
    const int64_t d = (int64_t)(jobs[b].k | 1) * jobs[b].n;
    if (d * 8 <= (int64_t)kBatchedSmem) need = std::max(need, d);
  }
  for (int b = count; b < kQrcpJobsPerLaunch; ++b) pj.j[b] = QrcpJob{};
  if (need > 0) {
    cudaError_t e = set_smem(qrcp_batched_kernel, (int)kBatchedSmem);
    if (e != cudaSuccess) return e;
  }
  qrcp_batched_kernel<<<count, kSmallThreads, (size_t)need * 8, st>>>(pj, tau, f, need);
  return cudaGetLastError();
}

cudaError_t launch_chol_update(const double *A, int64_t n, int64_t lda, const int64_t *rank,
                               double *Rp, int64_t ldrp, double *R, int64_t ldr,
                               int *dev_status, cudaStream_t st) {
  const size_t bytes = (size_t)(n | 1) * n * 8;
  const bool sm = bytes <= kCholSmem;
  if (sm) {
    cudaError_t e = set_smem(chol_factor_kernel, (int)kCholSmem);
    if (e != cudaSuccess) return e;
  }
  chol_factor_kernel<<<1, kSmallThreads, sm ? bytes : 0, st>>>(A, (int)n, lda, rank, Rp, ldrp, dev_status, sm);
  chol_apply_kernel<<<(unsigned)n, kApplyThreads, 0, st>>>(Rp, (int)n, ldrp, rank, R, ldr);
  return cudaGetLastError();
}

cudaError_t launch_tri_inverse(const double *R, int64_t n, int64_t ldr, const int64_t *rank,
                               double *W, int64_t ldw, cudaStream_t st) {
  tri_inverse_kernel<<<1, 256, 0, st>>>(R, (int)n, ldr, rank, W, ldw);
  return cudaGetLastError();
}

cudaError_t launch_reset_status(int *dev_status, cudaStream_t st) {
  reset_status_kernel<<<1, 1, 0, st>>>(dev_status);
  return cudaGetLastError();
}

cudaError_t launch_set_rank(int64_t *rank, int64_t value, cudaStream_t st) {
  set_rank_kernel<<<1, 1, 0, st>>>(rank, value);
  return cudaGetLastError();
}

}  // namespace rcqr
