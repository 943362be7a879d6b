/*
 * rcqr.h -- C ABI of librcqr.so: randomized Cholesky QR of a tall-skinny matrix
 * on one GB300 (sm_103a).
 *
 * Method: O. Balabanov, "Randomized Cholesky QR factorizations" (arXiv 2210.09953).
 * The problem (Sec. 1): X (m x n, n << m) = Q R with R upper triangular (or
 * trapezoidal, with permuted columns) and Q well conditioned or orthonormal.
 *
 * Conventions for every entry point
 *   - Matrices are column-major: element (i, j) of A lives at A[i + j * lda].
 *   - Every array argument is a DEVICE pointer owned by the caller, unless the
 *     comment says "host".  The library never allocates device memory, never
 *     frees caller memory and never synchronises the stream: scratch space is
 *     the caller's `workspace` (at least rcqr_workspace_size() bytes, 256-byte
 *     aligned), and all work is queued on `stream` in order.
 *   - Argument errors are returned synchronously (RCQR_EINVAL, RCQR_EWORKSPACE,
 *     RCQR_EUNSUPPORTED) before anything is queued.  A CUDA launch error gives
 *     RCQR_ECUDA.  Numerical failures found on the device (a Cholesky pivot
 *     <= 0, a zero sketch) are written to `dev_status` (device int[2]: status
 *     code, then the failing pivot index or -1), which the caller reads after
 *     synchronising; the entry points that take `dev_status` reset it first.
 *   - Theta (Sec. 2) is never stored.  Entry (i, r) of the k x m sketching
 *     matrix -- i < k, r the global row index of X -- is T[t] / sqrt(k v): t is
 *     byte (r mod 16) of Philox4x32-10(counter = (floor(r/16) mod 2^32,
 *     floor(r/16) div 2^32, i, stream), key = (seed mod 2^32, seed div 2^32)),
 *     T[t] = round(44 Phi^{-1}((t + 1/2)/256)) in [-127, 127] (the 256-point
 *     quantile grid of N(0,1)), v = (1/256) sum_t T[t]^2.  stream = 0 except in
 *     the batched call, where it is the problem index.
 *   - Precision `prec`: RCQR_F64 (X and Q are double), RCQR_F32 (X and Q are
 *     float), RCQR_BF16 (X is bfloat16, Q is float).  R, P, S, Z are always
 *     double.  The sketch and the small factorizations run in FP64-level
 *     precision for every prec (the multi-precision model of Sec. 1.3 and Sec. 5:
 *     the minor operations in higher precision).
 *   - Limits: 1 <= n <= 256, n <= k <= 2048, k a multiple of 8, m >= 1,
 *     ld >= m, 0 <= row_offset.
 */
#ifndef RCQR_H
#define RCQR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *cudaStream_t;

typedef enum {
  RCQR_OK = 0,
  RCQR_EINVAL = -1,       /* bad argument (sizes, leading dimensions, null pointer) */
  RCQR_ENOTSPD = -2,      /* device: Cholesky pivot <= 0 in the CholeskyQR pass (Alg. 3 step 3) */
  RCQR_ERANK0 = -3,       /* device: the sketch is zero, no column can be kept (Alg. 7 step 3) */
  RCQR_ECUDA = -4,        /* a CUDA call failed */
  RCQR_ETIMEOUT = -5,     /* device: a bounded wait inside a kernel gave up */
  RCQR_EWORKSPACE = -6,   /* workspace missing, too small or misaligned */
  RCQR_EUNSUPPORTED = -7  /* valid request this build does not support (e.g. no sm_103a device) */
} rcqr_status;

typedef enum {
  RCQR_DIRECT = 0,   /* RCholeskyQR, Alg. 2: Q well conditioned */
  RCQR_DIRECT2 = 1,  /* RCholeskyQR2, Alg. 3: Q orthonormal */
  RCQR_RR = 2,       /* RRRCholQR, Alg. 7 with the column normalisation of Sec. 4;
                        RRQR of step 2 = column-pivoted Householder QR */
  RCQR_RR2 = 3,      /* RRRCholQR followed by one CholeskyQR pass (Sec. 4) */
  RCQR_SRR = 4,      /* RRRCholQR whose RRQR is the strong rank-revealing QR of Gu and
                        Eisenstat with f = 1.5 (Sec. 4, Sec. 6.1; see rcqr_srrqr) */
  RCQR_SRR2 = 5      /* RCQR_SRR followed by one CholeskyQR pass */
} rcqr_variant;

typedef enum { RCQR_F64 = 0, RCQR_F32 = 1, RCQR_BF16 = 2 } rcqr_prec;

/* The distribution of Theta's entries (Sec. 2: Gaussian and Rademacher embeddings).
 * RCQR_THETA_GAUSSIAN: the 256-level quantile table described above (the default of
 * every call without a `theta` argument).  RCQR_THETA_RADEMACHER: entry (i, r) =
 * (1 - 2 b) / sqrt(k) with b = bit (r mod 128) of Philox4x32-10(counter =
 * (floor(r/128) mod 2^32, floor(r/128) div 2^32, i, stream), key = (seed mod 2^32,
 * seed div 2^32)), bit b of the 128-bit output being bit (b mod 32) of word
 * floor(b/32): one Philox bit per entry.  RCQR_THETA_SRHT: the subsampled randomized
 * Hadamard transform sqrt(1/k) S H D of Sec. 2, X padded with zero rows to 2^64 rows:
 * entry (i, r) = (1 - 2 s_r) (-1)^popcount(h_i AND r) / sqrt(k), where s_r is the
 * Rademacher bit above taken at the row index i = 2^32 - 1 (the random signs D, the same
 * for every row of Theta) and h_i = w0 + 2^32 w1, (w0, w1) the first two words of
 * Philox4x32-10(counter = (i, 0, 2^32 - 2, stream), same key): uniform sampling S of the
 * rows of the Sylvester-Hadamard matrix H, with replacement.  It is applied as the dense
 * +-1 product, exactly like the Rademacher one. */
typedef enum { RCQR_THETA_GAUSSIAN = 0, RCQR_THETA_RADEMACHER = 1, RCQR_THETA_SRHT = 2 } rcqr_theta;

/* Diagnostics: the bound of every device-side wait in the tensor-core
 * sketch's pipeline, in rounds of one mbarrier poll and a sleep of at most
 * 256 ns, for all later calls of this process; 0 restores the default of 2^22
 * rounds (about one second).  A wait that runs out stops the kernel from
 * issuing further tensor-core work; the kernel then waits (always with the
 * default bound) for the work already issued, writes NaN partial sums and sets
 * dev_status = {RCQR_ETIMEOUT, -1}.  Returns the previous bound.  Host-side and
 * not stream-ordered: change it only while no sketch is queued. */
uint32_t rcqr_set_wait_polls(uint32_t polls);

/* Diagnostics (the paper has no counterpart): throughput probes for the rooflines of
 * arithmetic-bound kernels.  rcqr_probe launches, on `stream`, one kernel of 4 CTAs of
 * 256 threads per SM that runs `iters` iterations of independent chains of one
 * operation kind and writes one checksum per thread to `scratch` (device, at least
 * rcqr_probe_scratch_bytes() bytes).  It returns the number of operations the kernel
 * performs (Philox4x32-10 calls, FP32 FMAs, FP64 FMAs or 32-bit integer multiply-adds),
 * or -1 on a bad argument or launch error; time the call with CUDA events on `stream`. */
typedef enum { RCQR_PROBE_PHILOX = 0, RCQR_PROBE_FFMA = 1, RCQR_PROBE_DFMA = 2, RCQR_PROBE_IMAD = 3 } rcqr_probe_kind;
size_t rcqr_probe_scratch_bytes(void);
int64_t rcqr_probe(int kind, int iters, void *scratch, size_t scratch_bytes, cudaStream_t stream);

/* Human-readable name of a status code (static string). */
const char *rcqr_status_string(int status);

/* Bytes of workspace rcqr_factor / rcqr_sketch and the other single-problem
 * calls need for these sizes (an upper bound valid for all of them, and for
 * rcqr_reduced with L = NULL). 0 on invalid sizes. */
size_t rcqr_workspace_size(int64_t m, int64_t n, int64_t k, int variant, int prec);

/* Bytes of workspace rcqr_reduced needs: l = the row count of an explicit
 * extractor L, or 0 for L = Theta (this also counts the l x n buffer of
 * Y = L X).  0 on invalid sizes. */
size_t rcqr_reduced_workspace_size(int64_t m, int64_t n, int64_t k, int64_t l, int prec);

/* Host: write the 256 integer levels T[t] of Theta (see above) to out[0..255].
 * Returns RCQR_OK. */
int rcqr_theta_table(int32_t *out);

/* Host: the scale c = 1/sqrt(k v) so that Theta = c * T[t]. */
double rcqr_theta_scale(int64_t k);

/* Sketch, Alg. 2 step 1 (Sec. 3.1: one pass over X, "a simple addition" as the
 * reduction):  P = Theta X  (k x n, double, ldp >= k), Theta's columns taken at
 * global rows row_offset .. row_offset+m-1, so sketches of row blocks of a
 * larger matrix add up to the sketch of the whole (the shard API).
 * colnorm2 (nullable, double[n]) receives the squared column norms of X
 * (the matrix D^2 of Sec. 4). */
rcqr_status rcqr_sketch(const void *X, int64_t m, int64_t n, int64_t ldx, int prec,
                        int64_t k, uint64_t seed, int64_t row_offset,
                        double *P, int64_t ldp, double *colnorm2,
                        void *workspace, size_t ws_bytes, cudaStream_t stream);

/* rcqr_sketch with the distribution of Theta chosen by `theta` (rcqr_theta). */
rcqr_status rcqr_sketch_theta(const void *X, int64_t m, int64_t n, int64_t ldx, int prec,
                              int64_t k, uint64_t seed, int theta, int64_t row_offset,
                              double *P, int64_t ldp, double *colnorm2,
                              void *workspace, size_t ws_bytes, cudaStream_t stream);

/* rcqr_sketch without a workspace argument, for callers that cannot provide
 * device scratch memory: a plugin whose fixed argument list has no room for a
 * workspace pointer, or code inside a host application that owns all device
 * memory through its own pool and forbids further allocations.  The paper has
 * no counterpart; it is a packaging choice of this library.
 * Same inputs and outputs as rcqr_sketch (row_offset included).  The partial
 * sums live in one 8 MiB array in the library's own device memory, which every
 * GPU that loads the library keeps until the process exits; this call never
 * allocates or frees memory.  The first call on each device looks the array's
 * address up, so make it before any stream capture on that device.  All calls
 * share the array: calls whose GPU work overlaps (streams not ordered with
 * each other) race on it.  Returns RCQR_EWORKSPACE when n*k (+ 2 x SM count x n
 * with colnorm2) exceeds the 2^20 doubles of the array, RCQR_EINVAL on bad
 * arguments. */
rcqr_status rcqr_sketch_noalloc(const void *X, int64_t m, int64_t n, int64_t ldx, int prec,
                                int64_t k, uint64_t seed, int64_t row_offset,
                                double *P, int64_t ldp, double *colnorm2, cudaStream_t stream);

/* Householder QR of a small k x n double matrix (Alg. 2 step 2, Sec. 3.1):
 * P = S R with S (k x n, orthonormal columns, nullable) and R (n x n, upper,
 * diag(R) >= 0, strictly lower part set to 0). */
rcqr_status rcqr_small_qr(const double *P, int64_t k, int64_t n, int64_t ldp,
                          double *S, int64_t lds, double *R, int64_t ldr,
                          void *workspace, size_t ws_bytes, cudaStream_t stream);

/* Column-pivoted Householder QR of P D^{-1} and the truncation rank (Alg. 7
 * steps 2-3, column normalisation of Sec. 4):  (P D^{-1})[:, perm] = S R,
 * D = diag(sqrt(colnorm2)) (colnorm2 nullable: D = I), pivot = the largest
 * recomputed remaining column norm, ties to the lowest index;
 * rank = min r with ||R[r:, r:]||_F <= tau ||R||_2; then R is overwritten by
 * R[:rank, :] Pi^T D Pi (rows >= rank set to 0).  perm: device int32[n];
 * rank: device int64.  dev_status gets RCQR_ERANK0 if rank = 0. */
rcqr_status rcqr_qrcp(const double *P, int64_t k, int64_t n, int64_t ldp,
                      const double *colnorm2, double tau,
                      double *R, int64_t ldr, int32_t *perm, int64_t *rank,
                      void *workspace, size_t ws_bytes, int *dev_status, cudaStream_t stream);

/* Strong rank-revealing QR for Alg. 7 steps 2-3 (the RRQR of Sec. 4 as Sec. 6.1 runs
 * it: Gu and Eisenstat's strong RRQR with parameter f, here after column pivoting).
 * Starts as rcqr_qrcp (same arguments and outputs), then, at the truncation rank r
 * (0 < r < n), swaps columns while some
 *   rho_ij = (R11^{-1} R12)_ij^2 + (gamma_j(R22) / omega_i(R11))^2 > f^2
 * (gamma_j = ||R22[:, j]||_2, omega_i = 1 / ||row i of R11^{-1}||_2; the largest rho_ij,
 * first in column-major order on ties), trading column i of the leading block with column
 * r + j and factoring P[:, perm] D^{-1} again (no pivoting).  Each swap multiplies
 * |det R11| by more than f; at most 4 n swaps per rank, and the rank test is repeated on
 * the swapped factor (at most 4 rounds while it changes).  On return every rho_ij <= f^2,
 * which gives sigma_i(R11) >= sigma_i(P D^{-1}) / q and sigma_j(R22) <= sigma_{r+j} q with
 * q = sqrt(1 + f^2 r (n - r)) (Gu and Eisenstat 1996, Thm. 3.2) -- the RRQR properties
 * the analysis of Sec. 5.3 assumes.  f >= 1; the variants RCQR_SRR/SRR2 use f = 1.5. */
rcqr_status rcqr_srrqr(const double *P, int64_t k, int64_t n, int64_t ldp, const double *colnorm2,
                       double tau, double f, double *R, int64_t ldr, int32_t *perm, int64_t *rank,
                       void *workspace, size_t ws_bytes, int *dev_status, cudaStream_t stream);

/* Forward substitution, Alg. 2 step 3:  Q = X R^{-1} (m x n; Q's type follows
 * prec: double for F64, float otherwise).  R is n x n upper with nonzero
 * diagonal.  perm (nullable device int32[n]) and rank (nullable device int64):
 * when given, the input columns are X[:, perm[j]] for j < rank and Q's columns
 * j >= rank are set to 0 (the RR form of Alg. 7 step 4).  Q may alias X only
 * when perm is NULL and the types match. */
rcqr_status rcqr_trsm(const void *X, int64_t m, int64_t n, int64_t ldx, int prec,
                      const double *R, int64_t ldr, const int32_t *perm, const int64_t *rank,
                      void *Q, int64_t ldq, void *workspace, size_t ws_bytes, cudaStream_t stream);

/* Alg. 2 step 3 and Alg. 3 step 2 in one pass over X (the first substitution of
 * RCholeskyQR2 with the Gram of its second pass): Q = X R^{-1} as in rcqr_trsm
 * and A = Q^T Q (n x n double, both triangles), without reading Q back.  Mixed
 * path only: prec RCQR_F32 or RCQR_BF16 (Q is float), n <= 64; otherwise
 * RCQR_EUNSUPPORTED.  perm/rank as in rcqr_trsm (A's columns >= rank are 0).
 * Q may not alias X.  workspace: rcqr_workspace_size(m, n, k, RCQR_DIRECT2, prec)
 * bytes for any valid k. */
rcqr_status rcqr_trsm_gram(const void *X, int64_t m, int64_t n, int64_t ldx, int prec,
                           const double *R, int64_t ldr, const int32_t *perm, const int64_t *rank,
                           float *Q, int64_t ldq, double *A, int64_t lda,
                           void *workspace, size_t ws_bytes, cudaStream_t stream);

/* Gram matrix, Alg. 3 step 2:  A = Q^T Q (n x n double, both triangles), Q of
 * type double (F64) or float (F32, BF16). rank (nullable): only the leading
 * rank x rank block is formed, the rest set to 0. */
rcqr_status rcqr_gram(const void *Q, int64_t m, int64_t n, int64_t ldq, int prec,
                      const int64_t *rank, double *A, int64_t lda,
                      void *workspace, size_t ws_bytes, cudaStream_t stream);

/* CholeskyQR update, Alg. 3 step 3:  R' = chol(A) (upper, positive diagonal),
 * R <- R' R.  R' is written to Rp (n x n, strictly lower part 0).  rank
 * (nullable): only the leading rank x rank block of A and rank rows of R are
 * used.  A pivot <= 0 sets dev_status = {RCQR_ENOTSPD, j} and leaves R as it was. */
rcqr_status rcqr_chol_update(const double *A, int64_t n, int64_t lda, const int64_t *rank,
                             double *Rp, int64_t ldrp, double *R, int64_t ldr,
                             int *dev_status, cudaStream_t stream);

/* The factorization (Alg. 2, 3, 7 and RRRCholQR2).
 * X: m x n (type by prec), Q: m x n (m x rank for RR; columns >= rank zeroed),
 * R: n x n double (RR: rows >= rank zeroed; X[:, perm] = Q R), perm: device
 * int32[n] (RR only, else nullable), rank: device int64 (nullable; n for the
 * direct variants).  tau: truncation tolerance of Alg. 7 step 3 (RR only).
 * Q may alias X for RCQR_DIRECT / RCQR_DIRECT2 when the types match. */
rcqr_status rcqr_factor(const void *X, int64_t m, int64_t n, int64_t ldx, int prec,
                        int64_t k, uint64_t seed, int variant, double tau,
                        void *Q, int64_t ldq, double *R, int64_t ldr,
                        int32_t *perm, int64_t *rank,
                        void *workspace, size_t ws_bytes, int *dev_status, cudaStream_t stream);

/* rcqr_factor with the distribution of Theta chosen by `theta` (rcqr_theta). */
rcqr_status rcqr_factor_theta(const void *X, int64_t m, int64_t n, int64_t ldx, int prec,
                              int64_t k, uint64_t seed, int theta, int variant, double tau,
                              void *Q, int64_t ldq, double *R, int64_t ldr,
                              int32_t *perm, int64_t *rank,
                              void *workspace, size_t ws_bytes, int *dev_status, cudaStream_t stream);

/* RCholeskyQR2 with an implicit Q factor (the remark after Alg. 3): Alg. 3 steps 1-3
 * only.  Q1 (m x n, Q's type by prec) receives the Q of Alg. 2, R the final R = R' R1,
 * Rp (n x n double, upper, diag > 0) the Cholesky factor R' of Q1^T Q1; the orthonormal
 * factor Q = Q1 R'^{-1} is never formed (one pass over the data fewer) and is applied
 * with rcqr_implicit_q_times / rcqr_implicit_qt_times.  Workspace and errors as
 * rcqr_factor with variant RCQR_DIRECT2. */
rcqr_status rcqr_factor_implicit(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, int64_t k,
                                 uint64_t seed, void *Q1, int64_t ldq, double *R, int64_t ldr, double *Rp,
                                 int64_t ldrp, void *workspace, size_t ws_bytes, int *dev_status,
                                 cudaStream_t stream);

/* Products of the implicit Q = Q1 R'^{-1} (prec RCQR_F64: Q1, Z/B double; RCQR_F32: float):
 *   rcqr_implicit_q_times:  Z = Q Y = Q1 (R'^{-1} Y), Y n x c double, Z m x c (Q1's type);
 *   rcqr_implicit_qt_times: Z = Q^T B = R'^{-T} (Q1^T B), B m x c (Q1's type), Z n x c double
 *     (the products summed in FP64 per row range, the ranges added in a fixed order).
 * Limits: n, c <= 256, n c <= 8192.  Workspace: rcqr_implicit_workspace_size(m, n, c). */
size_t rcqr_implicit_workspace_size(int64_t m, int64_t n, int64_t c);
rcqr_status rcqr_implicit_q_times(const void *Q1, int64_t m, int64_t n, int64_t ldq, int prec, const double *Rp,
                                  int64_t ldrp, const double *Y, int64_t ldy, int64_t c, void *Z, int64_t ldz,
                                  void *workspace, size_t ws_bytes, cudaStream_t stream);
rcqr_status rcqr_implicit_qt_times(const void *Q1, int64_t m, int64_t n, int64_t ldq, int prec, const double *Rp,
                                   int64_t ldrp, const void *B, int64_t ldb, int64_t c, double *Z, int64_t ldz,
                                   void *workspace, size_t ws_bytes, cudaStream_t stream);

/* Column-oriented RCholeskyQR, Alg. 4 (Sec. 3.2), one block of columns per call, for X
 * whose columns arrive in blocks (e.g. a Krylov basis built from the previous Q):
 * block i is the m x b matrix Xi, holding columns i0 .. i0+b-1 of X; Q (m x n, Q's
 * type by prec), S (k x n double) and R (n x n double) hold the earlier blocks' results
 * (columns < i0; R's leading i0 x i0 block).  The call computes
 *   P_i = Theta Xi;  R[:i0, i0:i0+b] = S[:, :i0]^+ P_i;
 *   [S_i, R_ii] = QR(P_i - S[:, :i0] R[:i0, i0:i0+b])  (S_i -> S[:, i0:i0+b], diag >= 0);
 *   Q[:, i0:i0+b] = (Xi - Q[:, :i0] R[:i0, i0:i0+b]) R_ii^{-1},
 * steps 3-4 as one Householder QR of the stacked [S[:, :i0] | P_i]; rows i0.. of R[:, :i0]
 * are set to 0.  rgs != 0: the randomized Gram-Schmidt form (remark after Alg. 4), S_i is
 * replaced by Theta Q_i.  Limits: 1 <= b <= 64, i0 + b <= min(256, k), k a multiple of 8.
 * Workspace: rcqr_colblock_workspace_size(m, b, k, i0, prec).  rcqr_factor_colwise runs
 * every block of a given X (widths b, the last one narrower) in order. */
size_t rcqr_colblock_workspace_size(int64_t m, int64_t b, int64_t k, int64_t i0, int prec);
rcqr_status rcqr_colblock_step(const void *Xi, int64_t m, int64_t b, int64_t ldx, int prec, int64_t k, uint64_t seed,
                               int64_t i0, int rgs, void *Q, int64_t ldq, double *S, int64_t lds, double *R,
                               int64_t ldr, void *workspace, size_t ws_bytes, int *dev_status, cudaStream_t stream);
rcqr_status rcqr_factor_colwise(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, int64_t k, uint64_t seed,
                                int64_t b, int rgs, void *Q, int64_t ldq, double *S, int64_t lds, double *R,
                                int64_t ldr, void *workspace, size_t ws_bytes, int *dev_status, cudaStream_t stream);

/* Reduced RCholeskyQR, Alg. 5:  P = Theta X, Y = L X, [S, R] = QR(P),
 * Z = Y R^{-1}.  L: l x m double extractor (ldl >= l), or NULL for L = Theta
 * (then l must equal k and Z = P R^{-1}, the sketch of Q).  Z: l x n,
 * S: k x n (nullable), R: n x n (diag(R) >= 0, the Householder R of P).
 * S is formed as P R^{-1} by substitution: the orthonormal factor of P up to
 * rounding amplified by cond(P) (the Householder S and P R^{-1} agree in exact
 * arithmetic).  Workspace: rcqr_reduced_workspace_size(m, n, k, L ? l : 0,
 * prec) bytes, checked before anything is queued. */
rcqr_status rcqr_reduced(const void *X, int64_t m, int64_t n, int64_t ldx, int prec,
                         int64_t k, uint64_t seed, const double *L, int64_t l, int64_t ldl,
                         double *Z, int64_t ldz, double *S, int64_t lds, double *R, int64_t ldr,
                         void *workspace, size_t ws_bytes, int *dev_status, cudaStream_t stream);

/* Reverse mode of RCholeskyQR2 (the paper has no counterpart: differentiation
 * is an addition of this library).  In exact arithmetic Alg. 3 returns the
 * unique thin QR of X (Q orthonormal, diag(R) > 0) whatever Theta is, so its
 * derivative is that of the thin QR map:
 *   M = R Rbar^T - Qbar^T Q,  Xbar = (Qbar + Q copyltu(M)) R^{-T},
 *   copyltu(M) = tril(M) + tril(M, -1)^T.
 * Q: the factor recomputed from X and the stored R (rcqr_trsm), m x n; Qbar
 * (same type as Q), Rbar (double, n x n, upper triangle used) the incoming
 * gradients; Xbar (type of Q) receives the gradient.  prec: RCQR_F64 (double
 * data, FP64) or RCQR_F32 (float data, FP32 rows with a compensated Qbar^T Q).
 * Workspace: rcqr_qr_adjoint_workspace_size(m, n) bytes (it holds an m x n buffer for
 * Y = Qbar + Q copyltu(M) besides the n x n matrices). */
size_t rcqr_qr_adjoint_workspace_size(int64_t m, int64_t n);
rcqr_status rcqr_qr_adjoint(const void *Q, int64_t m, int64_t n, int64_t ldq, int prec, const double *R,
                            int64_t ldr, const void *Qbar, int64_t ldqb, const double *Rbar, int64_t ldrb,
                            void *Xbar, int64_t ldxb, void *workspace, size_t ws_bytes, cudaStream_t stream);

/* One problem of a batched call (all pointers device, owned by the caller;
 * the fields mean what the arguments of the same names mean in rcqr_factor;
 * dev_status is this problem's device int[2]). */
typedef struct {
  const void *X;
  int64_t m, n, ldx, k;
  uint64_t seed;
  void *Q;
  int64_t ldq;
  double *R;
  int64_t ldr;
  int32_t *perm;   /* RR variants only, else nullable */
  int64_t *rank;   /* nullable */
  int *dev_status;
} rcqr_problem;

/* Workspace bytes for rcqr_factor_batched on these problems (host array). 0 on
 * invalid sizes. */
size_t rcqr_batched_workspace_size(const rcqr_problem *probs, int count, int variant, int prec);

/* Many factorizations (rcqr_factor, same variant, precision and tau for all)
 * of uneven sizes in one stream-ordered call: `probs` is a HOST array of count
 * problems; problem i uses Theta with Philox stream index i.  The problems are
 * spread over library-owned streams forked from `stream` by an event and
 * joined back, so the call can be recorded by a stream capture on `stream`
 * (make the first call on a device before capturing: it creates the streams).
 * Calls from several host threads on one device take turns (a per-device
 * lock is held from the fork to the join). Problem i's arguments are read from
 * the host array when the call is made; the array may be reused once the call
 * returns (a graph captured from the call keeps the values it saw).  Q must not alias X.  Argument errors of any problem
 * return RCQR_EINVAL before anything is queued. */
rcqr_status rcqr_factor_batched(const rcqr_problem *probs, int count, int variant, int prec, double tau,
                                void *workspace, size_t ws_bytes, cudaStream_t stream);

/* Time rcqr_factor_batched on these problems for 1, 2, 4, 8 and 16 streams
 * (synchronises `stream`), keep the fastest for later calls on this device and
 * write it to the JSON file named by the environment variable RCQR_TUNE_CACHE
 * when that is set (read back by later processes).  *best_streams (host)
 * receives the choice. */
rcqr_status rcqr_tune_batched(const rcqr_problem *probs, int count, int variant, int prec, double tau,
                              void *workspace, size_t ws_bytes, cudaStream_t stream, int *best_streams);

#ifdef __cplusplus
}
#endif
#endif /* RCQR_H */
