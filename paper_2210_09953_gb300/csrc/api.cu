// The C ABI of librcqr.so (declared in include/rcqr.h): argument checks,
// workspace layout and the stream-ordered sequence of kernels for each
// variant of the method.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "rcqr_internal.h"

namespace rcqr {

int num_sms() {
  static int count[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (count[dev] == 0) {
    int c = 0;
    if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0)
      c = 148;
    count[dev] = c;
  }
  return count[dev];
}

cudaError_t ensure_smem(const void *func, int bytes) {
  static std::mutex mu;
  static std::vector<std::pair<std::pair<const void *, int>, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  for (auto &d : done)
    if (d.first.first == func && d.first.second == dev && d.second >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.push_back({{func, dev}, bytes});
  return e;
}

namespace {

bool valid_prec(int prec) { return prec == RCQR_F64 || prec == RCQR_F32 || prec == RCQR_BF16; }

bool valid_theta(int theta) {
  return theta == RCQR_THETA_GAUSSIAN || theta == RCQR_THETA_RADEMACHER || theta == RCQR_THETA_SRHT;
}

bool valid_sizes(int64_t m, int64_t n, int64_t k) {
  return m >= 1 && n >= 1 && n <= 256 && k >= n && k <= 2048 && (k % 8) == 0;
}

bool aligned(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 255) == 0; }

rcqr_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return RCQR_OK;
  if (e == cudaErrorMemoryAllocation) return RCQR_EWORKSPACE;
  return RCQR_ECUDA;
}

// Workspace layout of rcqr_factor (the measuring pass uses the same code).
struct FactorBuffers {
  double *P, *R0, *A, *Rp, *colnorm2;
  int64_t *rank_tmp;
};

bool take_factor_buffers(Workspace &w, int64_t n, int64_t k, FactorBuffers &b) {
  b.P = w.take<double>((size_t)k * n);
  b.R0 = w.take<double>((size_t)n * n);
  b.A = w.take<double>((size_t)n * n);
  b.Rp = w.take<double>((size_t)n * n);
  b.colnorm2 = w.take<double>((size_t)n);
  b.rank_tmp = w.take<int64_t>(1);
  return w.ok();
}

size_t stage_workspace(int64_t m, int64_t n, int64_t k, int prec) {
  size_t s = sketch_workspace(m, n, k, 0, prec);
  s = std::max(s, small_qr_workspace(k, n));
  s = std::max(s, gram_workspace(m, n));
  s = std::max(s, trsm_workspace(m, n, prec));
  if (prec != RCQR_F64 && trsm32_gram_supported(n)) s = std::max(s, trsm32_gram_workspace(m, n));
  s = std::max(s, (size_t)n * n * 8 + 256);
  return s;
}

}  // namespace
}  // namespace rcqr

using namespace rcqr;

extern "C" {

const char *rcqr_status_string(int s) {
  switch (s) {
    case RCQR_OK: return "RCQR_OK";
    case RCQR_EINVAL: return "RCQR_EINVAL: invalid argument";
    case RCQR_ENOTSPD: return "RCQR_ENOTSPD: Cholesky pivot <= 0 in the CholeskyQR pass";
    case RCQR_ERANK0: return "RCQR_ERANK0: zero sketch, rank 0";
    case RCQR_ECUDA: return "RCQR_ECUDA: CUDA error";
    case RCQR_ETIMEOUT: return "RCQR_ETIMEOUT: bounded device wait expired";
    case RCQR_EWORKSPACE: return "RCQR_EWORKSPACE: workspace missing, too small or misaligned";
    case RCQR_EUNSUPPORTED: return "RCQR_EUNSUPPORTED: unsupported request";
    default: return "unknown rcqr status";
  }
}

int rcqr_theta_table(int32_t *out) {
  if (!out) return RCQR_EINVAL;
  const ThetaTable &t = theta_table();
  for (int i = 0; i < 256; ++i) out[i] = t.level[i];
  return RCQR_OK;
}

double rcqr_theta_scale(int64_t k) { return k > 0 ? theta_scale(k) : 0.0; }

size_t rcqr_workspace_size(int64_t m, int64_t n, int64_t k, int variant, int prec) {
  if (!valid_sizes(m, n, k) || !valid_prec(prec) || variant < 0 || variant > 5) return 0;
  Workspace w(nullptr, 0);
  FactorBuffers b;
  take_factor_buffers(w, n, k, b);
  const size_t fixed = w.used;
  size_t extra = stage_workspace(m, n, k, prec);
  extra = std::max(extra, dense_left_workspace(std::max<int64_t>(k, 1), m, n));
  return ((fixed + 255) & ~size_t(255)) + extra + 512;
}

rcqr_status rcqr_sketch_theta(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, int64_t k,
                              uint64_t seed, int theta, int64_t row_offset, double *P, int64_t ldp,
                              double *colnorm2, void *workspace, size_t ws_bytes, cudaStream_t stream) {
  if (!X || !P || !valid_prec(prec) || !valid_sizes(m, n, k) || ldx < m || ldp < k ||
      row_offset < 0 || !valid_theta(theta))
    return RCQR_EINVAL;
  if (!workspace || !aligned(workspace) || ws_bytes < sketch_workspace(m, n, k, row_offset, prec))
    return RCQR_EWORKSPACE;
  Workspace w(workspace, ws_bytes);
  return cuda_status(
      launch_sketch(X, m, n, ldx, prec, k, seed, 0, row_offset, P, ldp, colnorm2, w, stream, nullptr, theta));
}

rcqr_status rcqr_sketch(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, int64_t k,
                        uint64_t seed, int64_t row_offset, double *P, int64_t ldp,
                        double *colnorm2, void *workspace, size_t ws_bytes, cudaStream_t stream) {
  return rcqr_sketch_theta(X, m, n, ldx, prec, k, seed, RCQR_THETA_GAUSSIAN, row_offset, P, ldp, colnorm2,
                           workspace, ws_bytes, stream);
}

rcqr_status rcqr_small_qr(const double *P, int64_t k, int64_t n, int64_t ldp, double *S,
                          int64_t lds, double *R, int64_t ldr, void *workspace, size_t ws_bytes,
                          cudaStream_t stream) {
  if (!P || !R || n < 1 || n > 256 || k < n || k > 2048 || ldp < k || ldr < n || (S && lds < k))
    return RCQR_EINVAL;
  if (!workspace || !aligned(workspace) || ws_bytes < small_qr_workspace(k, n)) return RCQR_EWORKSPACE;
  Workspace w(workspace, ws_bytes);
  // S wanted: one CTA forms the reflectors and S; R only: the TSQR tree
  if (S) return cuda_status(launch_small_qr(P, k, n, ldp, S, lds, R, ldr, w, stream));
  return cuda_status(launch_small_r(P, k, n, ldp, R, ldr, w, stream));
}

rcqr_status rcqr_qrcp(const double *P, int64_t k, int64_t n, int64_t ldp, const double *colnorm2,
                      double tau, double *R, int64_t ldr, int32_t *perm, int64_t *rank,
                      void *workspace, size_t ws_bytes, int *dev_status, cudaStream_t stream) {
  if (!P || !R || !perm || !rank || n < 1 || n > 256 || k < n || k > 2048 || ldp < k || ldr < n ||
      !(tau >= 0.0))
    return RCQR_EINVAL;
  if (!workspace || !aligned(workspace) || ws_bytes < small_qr_workspace(k, n)) return RCQR_EWORKSPACE;
  Workspace w(workspace, ws_bytes);
  if (dev_status) {
    rcqr_status s = cuda_status(launch_reset_status(dev_status, stream));
    if (s != RCQR_OK) return s;
  }
  return cuda_status(
      launch_qrcp(P, k, n, ldp, colnorm2, tau, R, ldr, perm, rank, dev_status, w, stream));
}

rcqr_status rcqr_srrqr(const double *P, int64_t k, int64_t n, int64_t ldp, const double *colnorm2,
                       double tau, double f, double *R, int64_t ldr, int32_t *perm, int64_t *rank,
                       void *workspace, size_t ws_bytes, int *dev_status, cudaStream_t stream) {
  if (!P || !R || !perm || !rank || n < 1 || n > 256 || k < n || k > 2048 || ldp < k || ldr < n ||
      !(tau >= 0.0) || !(f >= 1.0))
    return RCQR_EINVAL;
  if (!workspace || !aligned(workspace) || ws_bytes < small_qr_workspace(k, n)) return RCQR_EWORKSPACE;
  Workspace w(workspace, ws_bytes);
  if (dev_status) {
    rcqr_status s = cuda_status(launch_reset_status(dev_status, stream));
    if (s != RCQR_OK) return s;
  }
  return cuda_status(
      launch_qrcp(P, k, n, ldp, colnorm2, tau, R, ldr, perm, rank, dev_status, w, stream, f));
}

rcqr_status rcqr_trsm(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, const double *R,
                      int64_t ldr, const int32_t *perm, const int64_t *rank, void *Q, int64_t ldq,
                      void *workspace, size_t ws_bytes, cudaStream_t stream) {
  if (!X || !R || !Q || !valid_prec(prec) || m < 1 || n < 1 || n > 256 || ldx < m || ldq < m ||
      ldr < n)
    return RCQR_EINVAL;
  if (perm && X == Q) return RCQR_EINVAL;
  if (X == Q && elem_size(prec) != q_elem_size(prec)) return RCQR_EINVAL;
  if (X == Q && ldx != ldq) return RCQR_EINVAL;
  const size_t need = trsm_workspace(m, n, prec);
  if (need > 0 && (!workspace || !aligned(workspace) || ws_bytes < need)) return RCQR_EWORKSPACE;
  Workspace w(workspace, ws_bytes);
  return cuda_status(launch_trsm(X, m, n, ldx, prec, R, ldr, perm, rank, Q, ldq, w, stream));
}

rcqr_status rcqr_trsm_gram(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, const double *R,
                           int64_t ldr, const int32_t *perm, const int64_t *rank, float *Q, int64_t ldq,
                           double *A, int64_t lda, void *workspace, size_t ws_bytes, cudaStream_t stream) {
  if (!X || !R || !Q || !A || !valid_prec(prec) || m < 1 || n < 1 || n > 256 || ldx < m || ldq < m ||
      ldr < n || lda < n || (const void *)Q == X)
    return RCQR_EINVAL;
  if (prec == RCQR_F64 || !trsm32_gram_supported(n)) return RCQR_EUNSUPPORTED;
  if (!workspace || !aligned(workspace) || ws_bytes < trsm32_gram_workspace(m, n)) return RCQR_EWORKSPACE;
  Workspace w(workspace, ws_bytes);
  return cuda_status(launch_trsm32_gram(X, m, n, ldx, prec, R, ldr, perm, rank, Q, ldq, A, lda, w, stream));
}

rcqr_status rcqr_gram(const void *Q, int64_t m, int64_t n, int64_t ldq, int prec,
                      const int64_t *rank, double *A, int64_t lda, void *workspace,
                      size_t ws_bytes, cudaStream_t stream) {
  if (!Q || !A || !valid_prec(prec) || m < 1 || n < 1 || n > 256 || ldq < m || lda < n)
    return RCQR_EINVAL;
  if (!workspace || !aligned(workspace) || ws_bytes < gram_workspace(m, n)) return RCQR_EWORKSPACE;
  Workspace w(workspace, ws_bytes);
  // Q's storage type: double for F64, float otherwise
  const int qprec = prec == RCQR_F64 ? RCQR_F64 : RCQR_F32;
  return cuda_status(launch_gram(Q, m, n, ldq, qprec, rank, A, lda, w, stream));
}

rcqr_status rcqr_chol_update(const double *A, int64_t n, int64_t lda, const int64_t *rank,
                             double *Rp, int64_t ldrp, double *R, int64_t ldr, int *dev_status,
                             cudaStream_t stream) {
  if (!A || !Rp || !R || n < 1 || n > 256 || lda < n || ldrp < n || ldr < n) return RCQR_EINVAL;
  if (dev_status) {
    rcqr_status s = cuda_status(launch_reset_status(dev_status, stream));
    if (s != RCQR_OK) return s;
  }
  return cuda_status(launch_chol_update(A, n, lda, rank, Rp, ldrp, R, ldr, dev_status, stream));
}

rcqr_status rcqr_factor(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, int64_t k,
                        uint64_t seed, int variant, double tau, void *Q, int64_t ldq, double *R,
                        int64_t ldr, int32_t *perm, int64_t *rank, void *workspace,
                        size_t ws_bytes, int *dev_status, cudaStream_t stream) {
  return rcqr::factor_impl(X, m, n, ldx, prec, k, seed, 0u, variant, tau, Q, ldq, R, ldr, perm, rank,
                           workspace, ws_bytes, dev_status, stream);
}

rcqr_status rcqr_factor_theta(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, int64_t k,
                              uint64_t seed, int theta, int variant, double tau, void *Q, int64_t ldq,
                              double *R, int64_t ldr, int32_t *perm, int64_t *rank, void *workspace,
                              size_t ws_bytes, int *dev_status, cudaStream_t stream) {
  if (!valid_theta(theta)) return RCQR_EINVAL;
  return rcqr::factor_impl(X, m, n, ldx, prec, k, seed, 0u, variant, tau, Q, ldq, R, ldr, perm, rank,
                           workspace, ws_bytes, dev_status, stream, theta);
}

}  // extern "C"

namespace rcqr {

// The factorization with Theta's Philox stream index (0 for single calls, the
// problem index in the batched call).
rcqr_status factor_impl(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, int64_t k,
                        uint64_t seed, uint32_t stream_id, int variant, double tau, void *Q,
                        int64_t ldq, double *R, int64_t ldr, int32_t *perm, int64_t *rank,
                        void *workspace, size_t ws_bytes, int *dev_status, cudaStream_t stream, int dist,
                        double *Rp_out, int64_t ldrp) {
  if (!X || !Q || !R || !dev_status || !valid_prec(prec) || !valid_sizes(m, n, k) || ldx < m ||
      ldq < m || ldr < n || variant < 0 || variant > 5)
    return RCQR_EINVAL;
  const bool rr = variant == RCQR_RR || variant == RCQR_RR2 || variant == RCQR_SRR || variant == RCQR_SRR2;
  const bool pass2 = variant == RCQR_DIRECT2 || variant == RCQR_RR2 || variant == RCQR_SRR2;
  // the strong-RRQR parameter f of Sec. 4 / Sec. 6.1 (0: column pivoting alone)
  const double strong_f = (variant == RCQR_SRR || variant == RCQR_SRR2) ? kStrongRrqrF : 0.0;
  if (rr && (!perm || !(tau >= 0.0))) return RCQR_EINVAL;
  if (X == Q && (rr || elem_size(prec) != q_elem_size(prec) || ldx != ldq)) return RCQR_EINVAL;
  if (!workspace || !aligned(workspace) || ws_bytes < rcqr_workspace_size(m, n, k, variant, prec))
    return RCQR_EWORKSPACE;

  Workspace w(workspace, ws_bytes);
  FactorBuffers b;
  if (!take_factor_buffers(w, n, k, b)) return RCQR_EWORKSPACE;
  const size_t mark = w.used;
  auto scratch = [&]() {
    w.used = mark;
    return &w;
  };
  int64_t *rk = rank ? rank : b.rank_tmp;
  const int qprec = prec == RCQR_F64 ? RCQR_F64 : RCQR_F32;

#define RCQR_TRY(expr)                              \
  do {                                              \
    rcqr_status _s = cuda_status(expr);             \
    if (_s != RCQR_OK) return _s;                   \
  } while (0)

  RCQR_TRY(launch_reset_status(dev_status, stream));
  // Alg. 2 / Alg. 7 step 1 (with D of Sec. 4 in the same pass for RR)
  RCQR_TRY(launch_sketch(X, m, n, ldx, prec, k, seed, stream_id, 0, b.P, k, rr ? b.colnorm2 : nullptr,
                         *scratch(), stream, dev_status, dist));
  const int32_t *pm = nullptr;
  const int64_t *rkp = nullptr;
  if (!rr) {
    // Alg. 2 step 2
    RCQR_TRY(launch_small_r(b.P, k, n, k, R, ldr, *scratch(), stream));
    RCQR_TRY(launch_set_rank(rk, n, stream));
  } else {
    // Alg. 7 steps 2-3 and the de-normalisation R <- R Pi^T D Pi
    RCQR_TRY(launch_qrcp(b.P, k, n, k, b.colnorm2, tau, R, ldr, perm, rk, dev_status, *scratch(),
                         stream, strong_f));
    pm = perm;
    rkp = rk;
  }
  // Alg. 2 step 3 / Alg. 7 step 4: for RR the leading block of the
  // de-normalised R is R11 D_sel, so Q = X Pi_{:,1:r} (R11 D_sel)^{-1}.
  const bool fused = pass2 && prec != RCQR_F64 && trsm32_gram_supported(n);
  if (fused) {
    // the substitution and the Gram of Alg. 3 step 2 in one pass over X
    RCQR_TRY(launch_trsm32_gram(X, m, n, ldx, prec, R, ldr, pm, rkp, (float *)Q, ldq, b.A, n, *scratch(),
                                stream, dev_status));
  } else {
    RCQR_TRY(launch_trsm(X, m, n, ldx, prec, R, ldr, pm, rkp, Q, ldq, *scratch(), stream, dev_status));
  }
  if (pass2) {
    // Alg. 3 steps 2-4 on the computed Q (implicit Q: steps 2-3 only, R' returned)
    if (!fused) RCQR_TRY(launch_gram(Q, m, n, ldq, qprec, rkp, b.A, n, *scratch(), stream));
    if (Rp_out)
      RCQR_TRY(launch_chol_update(b.A, n, n, rkp, Rp_out, ldrp, R, ldr, dev_status, stream));
    else
      RCQR_TRY(launch_cholqr_pass(b.A, n, rkp, b.Rp, R, ldr, Q, m, ldq, qprec, *scratch(), stream, dev_status));
  }
#undef RCQR_TRY
  return RCQR_OK;
}

}  // namespace rcqr

extern "C" {

size_t rcqr_qr_adjoint_workspace_size(int64_t m, int64_t n) {
  if (m < 1 || n < 1 || n > 256) return 0;
  return adjoint_workspace(m, n) + 256;
}

rcqr_status rcqr_qr_adjoint(const void *Q, int64_t m, int64_t n, int64_t ldq, int prec, const double *R,
                            int64_t ldr, const void *Qbar, int64_t ldqb, const double *Rbar, int64_t ldrb,
                            void *Xbar, int64_t ldxb, void *workspace, size_t ws_bytes, cudaStream_t stream) {
  if (!Q || !R || !Qbar || !Rbar || !Xbar || !(prec == RCQR_F64 || prec == RCQR_F32) || m < 1 || n < 1 ||
      n > 256 || ldq < m || ldqb < m || ldxb < m || ldr < n || ldrb < n)
    return RCQR_EINVAL;
  if (!workspace || !aligned(workspace) || ws_bytes < adjoint_workspace(m, n)) return RCQR_EWORKSPACE;
  Workspace w(workspace, ws_bytes);
  return cuda_status(launch_qr_adjoint(Q, m, n, ldq, prec, R, ldr, Qbar, ldqb, Rbar, ldrb, Xbar, ldxb, w, stream));
}

// Workspace of rcqr_reduced: the factor buffers, Y = L X (explicit L only), then the
// scratch of the sketch / small QR / substitution / dense left product.
size_t reduced_workspace(int64_t m, int64_t n, int64_t k, int64_t l, int prec) {
  Workspace w(nullptr, 0);
  FactorBuffers b;
  take_factor_buffers(w, n, k, b);
  if (l > 0) w.take<double>((size_t)l * n);
  size_t extra = stage_workspace(m, n, k, prec);
  if (l > 0) extra = std::max(extra, dense_left_workspace(l, m, n));
  return ((w.used + 255) & ~size_t(255)) + extra + 512;
}

size_t rcqr_reduced_workspace_size(int64_t m, int64_t n, int64_t k, int64_t l, int prec) {
  if (!valid_sizes(m, n, k) || !valid_prec(prec) || l < 0 || l > 2048) return 0;
  return reduced_workspace(m, n, k, l, prec);
}

rcqr_status rcqr_reduced(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, int64_t k,
                         uint64_t seed, const double *L, int64_t l, int64_t ldl, double *Z,
                         int64_t ldz, double *S, int64_t lds, double *R, int64_t ldr,
                         void *workspace, size_t ws_bytes, int *dev_status, cudaStream_t stream) {
  if (!X || !Z || !R || !valid_prec(prec) || !valid_sizes(m, n, k) || ldx < m || ldr < n ||
      (S && lds < k))
    return RCQR_EINVAL;
  if (L == nullptr && l != k) return RCQR_EINVAL;
  if (L != nullptr && (l < 1 || l > 2048 || ldl < l)) return RCQR_EINVAL;
  if (ldz < l) return RCQR_EINVAL;
  // every size check happens here, before anything is queued
  if (!workspace || !aligned(workspace) || ws_bytes < reduced_workspace(m, n, k, L ? l : 0, prec))
    return RCQR_EWORKSPACE;
  Workspace w(workspace, ws_bytes);
  FactorBuffers b;
  if (!take_factor_buffers(w, n, k, b)) return RCQR_EWORKSPACE;
  double *Y = nullptr;
  if (L) {
    Y = w.take<double>((size_t)l * n);
    if (!Y) return RCQR_EWORKSPACE;
  }
  const size_t mark = w.used;
  auto scratch = [&]() {
    w.used = mark;
    return &w;
  };
#define RCQR_TRY(expr)                              \
  do {                                              \
    rcqr_status _s = cuda_status(expr);             \
    if (_s != RCQR_OK) return _s;                   \
  } while (0)
  if (dev_status) RCQR_TRY(launch_reset_status(dev_status, stream));
  // Alg. 5 step 1
  RCQR_TRY(launch_sketch(X, m, n, ldx, prec, k, seed, 0, 0, b.P, k, nullptr, *scratch(), stream, dev_status));
  if (L) RCQR_TRY(launch_dense_left(L, l, ldl, X, m, n, ldx, prec, Y, l, *scratch(), stream));
  // Alg. 5 step 2: R of P = S R (the multi-CTA Householder R); S = P R^{-1}, the
  // orthonormal sketch of Q = X R^{-1}, by substitution against that R
  RCQR_TRY(launch_small_r(b.P, k, n, k, R, ldr, *scratch(), stream));
  if (S) RCQR_TRY(launch_trsm(b.P, k, n, k, RCQR_F64, R, ldr, nullptr, nullptr, S, lds, *scratch(), stream));
  // Alg. 5 step 3: Z = Y R^{-1} (Y = P when L = Theta)
  RCQR_TRY(launch_trsm(L ? Y : b.P, l, n, l, RCQR_F64, R, ldr, nullptr, nullptr, Z, ldz, *scratch(), stream));
#undef RCQR_TRY
  return RCQR_OK;
}

uint32_t rcqr_set_wait_polls(uint32_t polls) { return set_wait_polls(polls); }

rcqr_status rcqr_factor_implicit(const void *X, int64_t m, int64_t n, int64_t ldx, int prec, int64_t k,
                                 uint64_t seed, void *Q1, int64_t ldq, double *R, int64_t ldr, double *Rp,
                                 int64_t ldrp, void *workspace, size_t ws_bytes, int *dev_status,
                                 cudaStream_t stream) {
  if (!Rp || ldrp < n) return RCQR_EINVAL;
  return rcqr::factor_impl(X, m, n, ldx, prec, k, seed, 0u, RCQR_DIRECT2, 0.0, Q1, ldq, R, ldr, nullptr, nullptr,
                           workspace, ws_bytes, dev_status, stream, RCQR_THETA_GAUSSIAN, Rp, ldrp);
}

size_t rcqr_implicit_workspace_size(int64_t m, int64_t n, int64_t c) {
  if (m < 1 || !implicit_sizes_ok(n, c)) return 0;
  return implicit_workspace(m, n, c) + 512;
}

rcqr_status rcqr_implicit_q_times(const void *Q1, int64_t m, int64_t n, int64_t ldq, int prec, const double *Rp,
                                  int64_t ldrp, const double *Y, int64_t ldy, int64_t c, void *Z, int64_t ldz,
                                  void *workspace, size_t ws_bytes, cudaStream_t stream) {
  if (!Q1 || !Rp || !Y || !Z || !(prec == RCQR_F64 || prec == RCQR_F32) || m < 1 || !implicit_sizes_ok(n, c) ||
      ldq < m || ldrp < n || ldy < n || ldz < m)
    return RCQR_EINVAL;
  if (!workspace || !aligned(workspace) || ws_bytes < implicit_workspace(m, n, c)) return RCQR_EWORKSPACE;
  Workspace w(workspace, ws_bytes);
  return cuda_status(launch_implicit_q_times(Q1, m, n, ldq, prec, Rp, ldrp, Y, ldy, c, Z, ldz, w, stream));
}

rcqr_status rcqr_implicit_qt_times(const void *Q1, int64_t m, int64_t n, int64_t ldq, int prec, const double *Rp,
                                   int64_t ldrp, const void *B, int64_t ldb, int64_t c, double *Z, int64_t ldz,
                                   void *workspace, size_t ws_bytes, cudaStream_t stream) {
  if (!Q1 || !Rp || !B || !Z || !(prec == RCQR_F64 || prec == RCQR_F32) || m < 1 || !implicit_sizes_ok(n, c) ||
      ldq < m || ldrp < n || ldb < m || ldz < n)
    return RCQR_EINVAL;
  if (!workspace || !aligned(workspace) || ws_bytes < implicit_workspace(m, n, c)) return RCQR_EWORKSPACE;
  Workspace w(workspace, ws_bytes);
  return cuda_status(launch_implicit_qt_times(Q1, m, n, ldq, prec, Rp, ldrp, B, ldb, c, Z, ldz, w, stream));
}

}  // extern "C"
