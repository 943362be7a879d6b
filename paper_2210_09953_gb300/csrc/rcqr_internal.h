// Internal declarations shared by the translation units of librcqr.so.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/rcqr.h"

namespace rcqr {

// Theta levels packed for kernel arguments (256 signed 8-bit integers).
struct ThetaTable {
  int8_t level[256];
};

// Host-side table (own inverse-CDF code; identical integers to the definition
// in rcqr.h) and the scale 1/sqrt(k v).
const ThetaTable &theta_table();
double theta_scale(int64_t k);

// Bump allocator over the caller's workspace.  With base == nullptr it only
// measures (used by rcqr_workspace_size), so sizes and layout agree.
struct Workspace {
  char *base;
  size_t cap;
  size_t used = 0;
  Workspace(void *b, size_t c) : base(static_cast<char *>(b)), cap(c) {}
  template <class T>
  T *take(size_t count) {
    size_t off = (used + 255) & ~size_t(255);
    used = off + count * sizeof(T);
    if (base == nullptr || used > cap) return nullptr;
    return reinterpret_cast<T *>(base + off);
  }
  bool ok() const { return base != nullptr && used <= cap; }
  // the same buffer with everything carved after `mark` released again
  Workspace &rewind(size_t mark) {
    used = mark;
    return *this;
  }
};

int num_sms();

// Bound of the device-side pipeline waits of the tensor-core kernels (rounds of
// one poll and a short sleep); set_wait_polls(0) restores the default (about 1 s).
uint32_t wait_polls();
uint32_t set_wait_polls(uint32_t polls);

// Raise a kernel's dynamic shared-memory limit on the current device, once:
// later calls (for instance inside a stream capture) make no CUDA call.
cudaError_t ensure_smem(const void *func, int bytes);
template <class K>
inline cudaError_t set_smem(K *kernel, int bytes) {
  return ensure_smem(reinterpret_cast<const void *>(kernel), bytes);
}

// rcqr_factor with Theta's Philox stream index (0 for single calls).
rcqr_status factor_impl(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, int64_t k,
                        uint64_t seed, uint32_t stream_id, int variant, double tau, void *Q,
                        int64_t ldq, double *R, int64_t ldr, int32_t *perm, int64_t *rank,
                        void *workspace, size_t ws_bytes, int *dev_status, cudaStream_t stream,
                        int dist = RCQR_THETA_GAUSSIAN, double *Rp_out = nullptr, int64_t ldrp = 0);

// f of the strong rank-revealing QR in the RCQR_SRR / RCQR_SRR2 variants (Sec. 4, Sec. 6.1).
constexpr double kStrongRrqrF = 1.5;

inline bool rank_revealing_variant(int v) { return v == RCQR_RR || v == RCQR_RR2 || v == RCQR_SRR || v == RCQR_SRR2; }

inline size_t elem_size(int prec) { return prec == RCQR_F64 ? 8 : (prec == RCQR_F32 ? 4 : 2); }
inline size_t q_elem_size(int prec) { return prec == RCQR_F64 ? 8 : 4; }

// ---- sketch (P = Theta X), FP64-exact accumulation --------------------------
// Number of per-CTA partial sketches the sketch kernel writes (workspace sizing).
int sketch_groups(int64_t m, int64_t n, int64_t k, int64_t row_offset);
size_t sketch_workspace(int64_t m, int64_t n, int64_t k, int64_t row_offset, int prec);
cudaError_t launch_sketch(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, int64_t k,
                          uint64_t seed, uint32_t stream_id, int64_t row_offset, double *P,
                          int64_t ldp, double *colnorm2, Workspace &ws, cudaStream_t st,
                          int *dev_status = nullptr, int dist = RCQR_THETA_GAUSSIAN);
// The exact tensor-core sketch (tcgen05): partial sums per CTA in the workspace;
// colnorm2 (nullable) receives the squared column norms from the same pass.
size_t sketch_tc_workspace(int64_t m, int64_t n, int64_t k, int64_t row_offset, int prec);
cudaError_t launch_sketch_tc(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, int64_t k,
                             uint64_t seed, uint32_t stream_id, int64_t row_offset, double *P,
                             int64_t ldp, double *colnorm2, int *dev_status, Workspace &ws, cudaStream_t st,
                             int dist = RCQR_THETA_GAUSSIAN);
// The same sketch with its partial sums in a caller-given device buffer of
// scratch_doubles doubles (fewer row groups when the buffer is small); no workspace.
cudaError_t launch_sketch_into(const void *X, int64_t m, int64_t n, int64_t ldx, int prec,
                               int64_t k, uint64_t seed, int64_t row_offset, double *P,
                               int64_t ldp, double *colnorm2, double *scratch,
                               size_t scratch_doubles, cudaStream_t st);
// Dense Y = L X (l x n double), L an explicit l x m double matrix.
cudaError_t launch_dense_left(const double *L, int64_t l, int64_t ldl, const void *X, int64_t m,
                              int64_t n, int64_t ldx, int prec, double *Y, int64_t ldy,
                              Workspace &ws, cudaStream_t st);
size_t dense_left_workspace(int64_t l, int64_t m, int64_t n);

// ---- small dense FP64 kernels (one CTA each) --------------------------------
size_t small_qr_workspace(int64_t k, int64_t n);
cudaError_t launch_small_qr(const double *P, int64_t k, int64_t n, int64_t ldp, double *S,
                            int64_t lds, double *R, int64_t ldr, Workspace &ws, cudaStream_t st);
// R only (diag >= 0) by a TSQR tree over several CTAs.
cudaError_t launch_small_r(const double *P, int64_t k, int64_t n, int64_t ldp, double *R, int64_t ldr,
                           Workspace &ws, cudaStream_t st);
// f > 0: the strong-RRQR swaps of Gu & Eisenstat with parameter f follow the pivoting.
cudaError_t launch_qrcp(const double *P, int64_t k, int64_t n, int64_t ldp, const double *colnorm2,
                        double tau, double *R, int64_t ldr, int32_t *perm, int64_t *rank,
                        int *dev_status, Workspace &ws, cudaStream_t st, double f = 0.0);
// One QRCP of a batch (the arguments of launch_qrcp, gwork: qrcp_work_doubles(k, n) doubles).
struct QrcpJob {
  const double *P;
  int k, n;
  int64_t ldp;
  const double *colnorm2;
  double *R;
  int64_t ldr;
  int32_t *perm;
  int64_t *rank;
  int *status;
  double *gwork;
};
constexpr int kQrcpJobsPerLaunch = 128;
size_t qrcp_work_doubles(int64_t k, int64_t n);
// Up to kQrcpJobsPerLaunch QRCPs in one launch, one CTA each.
cudaError_t launch_qrcp_jobs(const QrcpJob *jobs, int count, double tau, cudaStream_t st, double f = 0.0);
// R' = chol(A[:r,:r]), R[:r,:] <- R' R[:r,:].
cudaError_t launch_chol_update(const double *A, int64_t n, int64_t lda, const int64_t *rank,
                               double *Rp, int64_t ldrp, double *R, int64_t ldr, int *dev_status,
                               cudaStream_t st);
// Alg. 3 steps 3-4: R' = chol(A), R <- R' R, Q <- Q R'^{-1} (in place).
cudaError_t launch_cholqr_pass(const double *A, int64_t n, const int64_t *rank, double *Rp, double *R, int64_t ldr,
                               void *Q, int64_t m, int64_t ldq, int qprec, Workspace &ws, cudaStream_t st,
                               int *dev_status);

// W = R^{-1} (n x n upper) for the leading rank x rank block (rank nullable).
// Q <- Q R'^{-1} for FP32 Q, 16 < n <= 128: W = R'^{-1} in FP64, then Q W on the tensor
// cores with an exact leading term (gemm_tc.cu); workspace gemm_tc_workspace(n).
bool gemm_tc_supported(int64_t n);
size_t gemm_tc_workspace(int64_t n);
cudaError_t launch_inverse_times(float *Q, int64_t m, int64_t n, int64_t ldq, const double *Rp, int64_t ldrp,
                                 const int64_t *rank, int *status, Workspace &ws, cudaStream_t st);
// A = Q^T Q for FP32 Q, 64 < n <= 128, on the tensor cores (gemm_tc.cu); workspace
// gram_tc_workspace(m, n).
bool gram_tc_supported(int64_t n);
size_t gram_tc_workspace(int64_t m, int64_t n);
cudaError_t launch_gram_tc(const float *Q, int64_t m, int64_t n, int64_t ldq, double *A, int64_t lda, int *status,
                           Workspace &ws, cudaStream_t st);
// Q = X R^{-1} for 64 < n <= 128, FP32 / BF16 X: blocked substitution with the
// off-diagonal products on the tensor cores (trsm_tcw.cu); Rf, dinv from trsm32_prep_kernel.
bool trsm_tcw_supported(int64_t n);
cudaError_t launch_trsm_tcw(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, const float *Rf,
                            const float *dinv, const int32_t *perm, const int64_t *rank, float *Q, int64_t ldq,
                            int *status, cudaStream_t st);
cudaError_t launch_tri_inverse(const double *R, int64_t n, int64_t ldr, const int64_t *rank,
                               double *W, int64_t ldw, cudaStream_t st);
cudaError_t launch_reset_status(int *dev_status, cudaStream_t st);
cudaError_t launch_set_rank(int64_t *rank, int64_t value, cudaStream_t st);

// ---- bulk kernels over m -----------------------------------------------------
size_t trsm_workspace(int64_t m, int64_t n, int prec);
cudaError_t launch_trsm(const void *X, int64_t m, int64_t n, int64_t ldx, int prec,
                        const double *R, int64_t ldr, const int32_t *perm, const int64_t *rank,
                        void *Q, int64_t ldq, Workspace &ws, cudaStream_t st,
                        int *dev_status = nullptr);
// FP32 substitution and Gram of the mixed path (trsm_f32.cu).
bool trsm32_supported(int64_t n);
size_t trsm32_workspace(int64_t n);
cudaError_t launch_trsm32(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, const double *R,
                          int64_t ldr, const int32_t *perm, const int64_t *rank, void *Q, int64_t ldq,
                          Workspace &ws, cudaStream_t st);
int gram32_groups(int64_t m, int64_t n);
cudaError_t launch_gram32(const float *Q, int64_t m, int64_t n, int64_t ldq, const int64_t *rank,
                          double *partial, int groups, cudaStream_t st);
// Substitution fused with the second pass's Gram (mixed path, n <= 64): writes Q
// and A = Q^T Q (FP64, lda).
bool trsm32_gram_supported(int64_t n);
size_t trsm32_gram_workspace(int64_t m, int64_t n);
cudaError_t launch_trsm32_gram(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, const double *R,
                               int64_t ldr, const int32_t *perm, const int64_t *rank, float *Q, int64_t ldq,
                               double *A, int64_t lda, Workspace &ws, cudaStream_t st, int *dev_status = nullptr);
// Blocked substitution on the tensor cores fused with the Gram (trsm_tc.cu), 32 < n <= 64:
// Rf is the 64 x 64 FP32 R of trsm32_prep_kernel; `partial` receives one n x n FP64 partial
// Gram matrix of Q per CTA (trsm_tc_gram_groups(m) of them).
bool trsm_tc_supported(int64_t n);
int trsm_tc_gram_groups(int64_t m);
cudaError_t launch_trsm_tc_gram(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, const float *Rf,
                                const float *dinv, const int32_t *perm, const int64_t *rank, float *Q, int64_t ldq,
                                double *partial, int *status, cudaStream_t st);
// The implicit Q of RCholeskyQR2 (implicit.cu): Z = Q1 (R'^{-1} Y) and Z = R'^{-T} (Q1^T B).
bool implicit_sizes_ok(int64_t n, int64_t c);
size_t implicit_workspace(int64_t m, int64_t n, int64_t c);
cudaError_t launch_implicit_q_times(const void *Q, int64_t m, int64_t n, int64_t ldq, int prec, const double *Rp,
                                    int64_t ldrp, const double *Y, int64_t ldy, int64_t c, void *Z, int64_t ldz,
                                    Workspace &ws, cudaStream_t st);
cudaError_t launch_implicit_qt_times(const void *Q, int64_t m, int64_t n, int64_t ldq, int prec, const double *Rp,
                                     int64_t ldrp, const void *B, int64_t ldb, int64_t c, double *Z, int64_t ldz,
                                     Workspace &ws, cudaStream_t st);
// Column-oriented RCholeskyQR, one block (colwise.cu).
bool colblock_sizes_ok(int64_t m, int64_t b, int64_t k, int64_t i0);
size_t colblock_workspace(int64_t m, int64_t b, int64_t k, int64_t i0, int prec);
cudaError_t colblock_step(const void *Xi, int64_t m, int64_t b, int64_t ldx, int prec, int64_t k, uint64_t seed,
                          int64_t i0, int rgs, void *Q, int64_t ldq, double *S, int64_t lds, double *R, int64_t ldr,
                          Workspace &ws, cudaStream_t st, int *dev_status);
// A = sum of `groups` n x n partials (fixed order), trsm_simt.cu.
cudaError_t launch_gram_reduce(const double *partial, int groups, int64_t n, double *A, int64_t lda,
                               cudaStream_t st);
// Reverse mode of the thin QR map (adjoint.cu).
size_t adjoint_workspace(int64_t m, int64_t n);
cudaError_t launch_qr_adjoint(const void *Q, int64_t m, int64_t n, int64_t ldq, int prec, const double *R,
                              int64_t ldr, const void *Qbar, int64_t ldqb, const double *Rbar, int64_t ldrb,
                              void *Xbar, int64_t ldxb, Workspace &ws, cudaStream_t st);
size_t gram_workspace(int64_t m, int64_t n);
cudaError_t launch_gram(const void *Q, int64_t m, int64_t n, int64_t ldq, int prec,
                        const int64_t *rank, double *A, int64_t lda, Workspace &ws,
                        cudaStream_t st);

}  // namespace rcqr
