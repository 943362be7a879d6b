// Batched factorizations: many tall-skinny problems of uneven m and n in one
// call, every launch stream-ordered so that a caller's stream capture records
// the whole batch as one CUDA graph.
//
// The problems are sorted by size (largest first) and dealt round-robin to a
// set of library-owned streams forked from the caller's stream by an event
// and joined back by events (under capture: a multi-branch graph).  Problem i
// uses Theta's Philox stream index i.
//
// The direct variants run rcqr_factor's steps per problem in its stream's
// slice of the workspace.  The rank-revealing variants run in three phases,
// because their column-pivoted QR (one CTA, FP64, latency-bound) would
// otherwise run at most one per stream: (A) every problem's status reset,
// column norms and sketch, on the streams, into a per-problem region of the
// workspace; (B) all the QRCPs, one CTA each, in launches of up to
// kQrcpJobsPerLaunch problems spread over the streams; (C) every problem's
// substitution (and, for RR2, the CholeskyQR pass), on the streams.
// rcqr_tune_batched times the batch for several stream counts and keeps the
// fastest per device (and in the JSON file named by RCQR_TUNE_CACHE, when set).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <numeric>
#include <vector>

#include "rcqr_internal.h"

namespace rcqr {

namespace {

constexpr int kMaxStreams = 16;

struct DevStreams {
  bool ready = false;
  cudaStream_t s[kMaxStreams];
  cudaEvent_t fork;
  cudaEvent_t join[kMaxStreams];
  // held from the fork to the join of one call: concurrent calls on one device
  // (from several host threads) take turns instead of interleaving their events
  std::mutex call_mu;
};

std::mutex g_mu;
DevStreams g_streams[64];
std::atomic<int> g_best_streams[64];

// Fork of the library streams from the caller's stream; the join back runs on
// every exit path (also after an error), so a stream capture on the caller's
// stream always ends with every forked branch joined.
struct ForkGuard {
  DevStreams *d;
  cudaStream_t stream;
  int n = 0;
  ForkGuard(DevStreams *dd, cudaStream_t st) : d(dd), stream(st) {}
  bool fork(int ns) {
    if (cudaEventRecord(d->fork, stream) != cudaSuccess) return false;
    for (int s2 = 0; s2 < ns; ++s2) {
      if (cudaStreamWaitEvent(d->s[s2], d->fork, 0) != cudaSuccess) {
        n = s2;
        return false;
      }
    }
    n = ns;
    return true;
  }
  bool join() {
    bool ok = true;
    for (int s2 = 0; s2 < n; ++s2) {
      ok = cudaEventRecord(d->join[s2], d->s[s2]) == cudaSuccess && ok;
      ok = cudaStreamWaitEvent(stream, d->join[s2], 0) == cudaSuccess && ok;
    }
    n = 0;
    return ok;
  }
  ~ForkGuard() {
    if (n) join();
  }
};

cudaError_t device_streams(DevStreams **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  DevStreams &d = g_streams[dev];
  if (!d.ready) {
    for (int i = 0; i < kMaxStreams; ++i) {
      if ((e = cudaStreamCreateWithFlags(&d.s[i], cudaStreamNonBlocking)) != cudaSuccess) return e;
      if ((e = cudaEventCreateWithFlags(&d.join[i], cudaEventDisableTiming)) != cudaSuccess) return e;
    }
    if ((e = cudaEventCreateWithFlags(&d.fork, cudaEventDisableTiming)) != cudaSuccess) return e;
    d.ready = true;
  }
  *out = &d;
  return cudaSuccess;
}

int default_streams(int count) {
  int dev = 0;
  cudaGetDevice(&dev);
  const int tuned = (dev >= 0 && dev < 64) ? g_best_streams[dev].load() : 0;
  int ns = tuned > 0 ? tuned : 8;
  if (const char *path = std::getenv("RCQR_TUNE_CACHE")) {
    if (tuned <= 0) {
      if (FILE *f = std::fopen(path, "r")) {
        int v = 0;
        if (std::fscanf(f, " { \"batched_streams\" : %d", &v) == 1 && v >= 1 && v <= kMaxStreams) ns = v;
        std::fclose(f);
      }
    }
  }
  return std::max(1, std::min(ns, std::min(count, kMaxStreams)));
}

bool valid_problem(const rcqr_problem &p, int variant, int prec) {
  if (!p.X || !p.Q || !p.R || !p.dev_status) return false;
  if (p.m < 1 || p.n < 1 || p.n > 256 || p.k < p.n || p.k > 2048 || (p.k % 8) != 0) return false;
  if (p.ldx < p.m || p.ldq < p.m || p.ldr < p.n) return false;
  if (rank_revealing_variant(variant) && !p.perm) return false;
  if (p.X == p.Q) return false;
  (void)prec;
  return true;
}

bool rank_revealing(int variant) { return rank_revealing_variant(variant); }

// Per-problem region of the rank-revealing phases: P (k x n), the squared column
// norms (n) and the QRCP working copy, each 256-byte aligned.
size_t rr_region_bytes(const rcqr_problem &p) {
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  return al((size_t)p.k * p.n * 8) + al((size_t)p.n * 8) + al(qrcp_work_doubles(p.k, p.n) * 8);
}

size_t rr_persist_bytes(const rcqr_problem *probs, int count) {
  size_t s = 0;
  for (int i = 0; i < count; ++i) s += rr_region_bytes(probs[i]);
  return s;
}

size_t slice_bytes(const rcqr_problem *probs, int count, int variant, int prec) {
  size_t s = 0;
  for (int i = 0; i < count; ++i)
    s = std::max(s, rcqr_workspace_size(probs[i].m, probs[i].n, probs[i].k, variant, prec));
  return (s + 255) & ~size_t(255);
}

rcqr_status run_batch_rr(const rcqr_problem *probs, int count, int variant, int prec, double tau, void *workspace,
                         size_t ws_bytes, cudaStream_t stream, int ns, DevStreams *d, const std::vector<int> &order) {
  const size_t slice = slice_bytes(probs, count, variant, prec);
  const size_t persist = rr_persist_bytes(probs, count);
  if (persist + (size_t)ns * slice > ws_bytes) return RCQR_EWORKSPACE;
  char *base = static_cast<char *>(workspace);
  char *slices = base + persist;
  std::vector<double *> Pp(count), cnp(count), gwp(count);
  {
    size_t off = 0;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    for (int i = 0; i < count; ++i) {
      const rcqr_problem &p = probs[i];
      Pp[i] = reinterpret_cast<double *>(base + off);
      off += al((size_t)p.k * p.n * 8);
      cnp[i] = reinterpret_cast<double *>(base + off);
      off += al((size_t)p.n * 8);
      gwp[i] = reinterpret_cast<double *>(base + off);
      off += al(qrcp_work_doubles(p.k, p.n) * 8);
    }
  }
  ForkGuard fg(d, stream);
  // (A) status, column norms and sketch
  if (!fg.fork(ns)) return RCQR_ECUDA;
  for (int t = 0; t < count; ++t) {
    const int i = order[t];
    const rcqr_problem &p = probs[i];
    cudaStream_t st = d->s[t % ns];
    Workspace w(slices + (size_t)(t % ns) * slice, slice);
    if (launch_reset_status(p.dev_status, st) != cudaSuccess) return RCQR_ECUDA;
    if (launch_sketch(p.X, p.m, p.n, p.ldx, prec, p.k, p.seed, (uint32_t)i, 0, Pp[i], p.k, cnp[i], w, st,
                      p.dev_status) != cudaSuccess)
      return RCQR_ECUDA;
  }
  if (!fg.join()) return RCQR_ECUDA;
  // (B) the QRCPs, one CTA each
  const int nlaunch = (count + kQrcpJobsPerLaunch - 1) / kQrcpJobsPerLaunch;
  const int nb = std::min(nlaunch, kMaxStreams);
  if (!fg.fork(nb)) return RCQR_ECUDA;
  std::vector<QrcpJob> jobs(count);
  for (int t = 0; t < count; ++t) {
    const int i = order[t];
    const rcqr_problem &p = probs[i];
    jobs[t] = QrcpJob{Pp[i], (int)p.k, (int)p.n, p.k, cnp[i], p.R, p.ldr, p.perm, p.rank, p.dev_status, gwp[i]};
  }
  for (int c = 0; c < nlaunch; ++c) {
    const int b0 = c * kQrcpJobsPerLaunch, cnt = std::min(kQrcpJobsPerLaunch, count - b0);
    const double f = (variant == RCQR_SRR || variant == RCQR_SRR2) ? kStrongRrqrF : 0.0;
    if (launch_qrcp_jobs(jobs.data() + b0, cnt, tau, d->s[c % nb], f) != cudaSuccess) return RCQR_ECUDA;
  }
  if (!fg.join()) return RCQR_ECUDA;
  // (C) substitution (Alg. 7 step 4) and, for RR2, one CholeskyQR pass (Alg. 3 steps 2-4)
  const bool pass2 = variant == RCQR_RR2 || variant == RCQR_SRR2;
  const int qprec = prec == RCQR_F64 ? RCQR_F64 : RCQR_F32;
  if (!fg.fork(ns)) return RCQR_ECUDA;
  for (int t = 0; t < count; ++t) {
    const int i = order[t];
    const rcqr_problem &p = probs[i];
    cudaStream_t st = d->s[t % ns];
    Workspace w(slices + (size_t)(t % ns) * slice, slice);
    double *A = w.take<double>((size_t)p.n * p.n);
    double *Rp = w.take<double>((size_t)p.n * p.n);
    if (!A || !Rp) return RCQR_EWORKSPACE;
    const size_t mark = w.used;
    cudaError_t e;
    const bool fused = pass2 && prec != RCQR_F64 && trsm32_gram_supported(p.n);
    if (fused)
      e = launch_trsm32_gram(p.X, p.m, p.n, p.ldx, prec, p.R, p.ldr, p.perm, p.rank, (float *)p.Q, p.ldq, A, p.n,
                             w.rewind(mark), st);
    else
      e = launch_trsm(p.X, p.m, p.n, p.ldx, prec, p.R, p.ldr, p.perm, p.rank, p.Q, p.ldq, w.rewind(mark), st,
                      p.dev_status);
    if (e != cudaSuccess) return RCQR_ECUDA;
    if (pass2) {
      if (!fused && launch_gram(p.Q, p.m, p.n, p.ldq, qprec, p.rank, A, p.n, w.rewind(mark), st) != cudaSuccess)
        return RCQR_ECUDA;
      if (launch_cholqr_pass(A, p.n, p.rank, Rp, p.R, p.ldr, p.Q, p.m, p.ldq, qprec, w.rewind(mark), st,
                             p.dev_status) != cudaSuccess)
        return RCQR_ECUDA;
    }
  }
  if (!fg.join()) return RCQR_ECUDA;
  return RCQR_OK;
}

rcqr_status run_batch(const rcqr_problem *probs, int count, int variant, int prec, double tau,
                      void *workspace, size_t ws_bytes, cudaStream_t stream, int ns) {
  DevStreams *d = nullptr;
  if (device_streams(&d) != cudaSuccess) return RCQR_ECUDA;
  const size_t slice = slice_bytes(probs, count, variant, prec);
  if (!rank_revealing(variant) && (size_t)ns * slice > ws_bytes) return RCQR_EWORKSPACE;
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return probs[a].m * probs[a].n > probs[b].m * probs[b].n;
  });
  std::lock_guard<std::mutex> call_lock(d->call_mu);
  if (rank_revealing(variant))
    return run_batch_rr(probs, count, variant, prec, tau, workspace, ws_bytes, stream, ns, d, order);
  ForkGuard fg(d, stream);
  if (!fg.fork(ns)) return RCQR_ECUDA;
  rcqr_status st = RCQR_OK;
  for (int t = 0; t < count && st == RCQR_OK; ++t) {
    const int i = order[t];
    const int s = t % ns;
    const rcqr_problem &p = probs[i];
    char *ws = static_cast<char *>(workspace) + (size_t)s * slice;
    st = factor_impl(p.X, p.m, p.n, p.ldx, prec, p.k, p.seed, (uint32_t)i, variant, tau, p.Q, p.ldq, p.R,
                     p.ldr, p.perm, p.rank, ws, slice, p.dev_status, d->s[s]);
  }
  if (!fg.join() && st == RCQR_OK) return RCQR_ECUDA;
  return st;
}

}  // namespace

}  // namespace rcqr

using namespace rcqr;

extern "C" {

size_t rcqr_batched_workspace_size(const rcqr_problem *probs, int count, int variant, int prec) {
  if (!probs || count < 1) return 0;
  for (int i = 0; i < count; ++i)
    if (rcqr_workspace_size(probs[i].m, probs[i].n, probs[i].k, variant, prec) == 0) return 0;
  const size_t persist = rank_revealing(variant) ? rr_persist_bytes(probs, count) : 0;
  return persist + (size_t)std::min(count, kMaxStreams) * slice_bytes(probs, count, variant, prec) + 256;
}

rcqr_status rcqr_factor_batched(const rcqr_problem *probs, int count, int variant, int prec, double tau,
                                void *workspace, size_t ws_bytes, cudaStream_t stream) {
  if (!probs || count < 1 || variant < 0 || variant > 5 || !(prec >= 0 && prec <= 2)) return RCQR_EINVAL;
  if (rank_revealing_variant(variant) && !(tau >= 0.0)) return RCQR_EINVAL;
  for (int i = 0; i < count; ++i)
    if (!valid_problem(probs[i], variant, prec)) return RCQR_EINVAL;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return RCQR_EWORKSPACE;
  return run_batch(probs, count, variant, prec, tau, workspace, ws_bytes, stream, default_streams(count));
}

rcqr_status rcqr_tune_batched(const rcqr_problem *probs, int count, int variant, int prec, double tau,
                              void *workspace, size_t ws_bytes, cudaStream_t stream, int *best_streams) {
  if (!probs || count < 1 || !best_streams) return RCQR_EINVAL;
  for (int i = 0; i < count; ++i)
    if (!valid_problem(probs[i], variant, prec)) return RCQR_EINVAL;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return RCQR_ECUDA;
  float best_ms = 1e30f;
  int best = 1;
  const int cands[5] = {1, 2, 4, 8, 16};
  for (int ci = 0; ci < 5; ++ci) {
    const int ns = std::min(cands[ci], std::min(count, kMaxStreams));
    if (ci > 0 && ns == std::min(cands[ci - 1], std::min(count, kMaxStreams))) continue;
    rcqr_status st = run_batch(probs, count, variant, prec, tau, workspace, ws_bytes, stream, ns);
    if (st != RCQR_OK) continue;
    cudaEventRecord(a, stream);
    for (int r = 0; r < 3 && st == RCQR_OK; ++r)
      st = run_batch(probs, count, variant, prec, tau, workspace, ws_bytes, stream, ns);
    cudaEventRecord(b, stream);
    if (cudaEventSynchronize(b) != cudaSuccess) {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      return RCQR_ECUDA;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (st == RCQR_OK && ms < best_ms) {
      best_ms = ms;
      best = ns;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64) g_best_streams[dev].store(best);
  if (const char *path = std::getenv("RCQR_TUNE_CACHE")) {
    if (FILE *f = std::fopen(path, "w")) {
      std::fprintf(f, "{ \"batched_streams\" : %d, \"ms_per_batch\" : %.4f }\n", best, best_ms / 3.0f);
      std::fclose(f);
    }
  }
  *best_streams = best;
  return RCQR_OK;
}

}  // extern "C"
