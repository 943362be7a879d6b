// Batched factorizations: many tall-skinny problems of uneven m and n in one
// call, every launch stream-ordered so that a caller's stream capture records
// the whole batch as one CUDA graph.
//
// The problems are sorted by size (largest first) and dealt round-robin to a
// set of library-owned streams forked from the caller's stream by an event
// and joined back by events (under capture: a multi-branch graph).  Each
// problem i runs the factorization of rcqr_factor with Theta's Philox stream
// index i, in its stream's slice of the workspace.  rcqr_tune_batched times
// the batch for several stream counts and keeps the fastest per device (and
// in the JSON file named by RCQR_TUNE_CACHE, when set).
#include <cuda_runtime.h>

#include <algorithm>
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
};

std::mutex g_mu;
DevStreams g_streams[64];
int g_best_streams[64] = {0};

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
  int ns = (dev >= 0 && dev < 64 && g_best_streams[dev] > 0) ? g_best_streams[dev] : 8;
  if (const char *path = std::getenv("RCQR_TUNE_CACHE")) {
    if (!(dev >= 0 && dev < 64 && g_best_streams[dev] > 0)) {
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
  if ((variant == RCQR_RR || variant == RCQR_RR2) && !p.perm) return false;
  if (p.X == p.Q) return false;
  (void)prec;
  return true;
}

size_t slice_bytes(const rcqr_problem *probs, int count, int variant, int prec) {
  size_t s = 0;
  for (int i = 0; i < count; ++i)
    s = std::max(s, rcqr_workspace_size(probs[i].m, probs[i].n, probs[i].k, variant, prec));
  return (s + 255) & ~size_t(255);
}

rcqr_status run_batch(const rcqr_problem *probs, int count, int variant, int prec, double tau,
                      void *workspace, size_t ws_bytes, cudaStream_t stream, int ns) {
  DevStreams *d = nullptr;
  if (device_streams(&d) != cudaSuccess) return RCQR_ECUDA;
  const size_t slice = slice_bytes(probs, count, variant, prec);
  if ((size_t)ns * slice > ws_bytes) return RCQR_EWORKSPACE;
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return probs[a].m * probs[a].n > probs[b].m * probs[b].n;
  });
  if (cudaEventRecord(d->fork, stream) != cudaSuccess) return RCQR_ECUDA;
  for (int s = 0; s < ns; ++s)
    if (cudaStreamWaitEvent(d->s[s], d->fork, 0) != cudaSuccess) return RCQR_ECUDA;
  rcqr_status st = RCQR_OK;
  for (int t = 0; t < count && st == RCQR_OK; ++t) {
    const int i = order[t];
    const int s = t % ns;
    const rcqr_problem &p = probs[i];
    char *ws = static_cast<char *>(workspace) + (size_t)s * slice;
    st = factor_impl(p.X, p.m, p.n, p.ldx, prec, p.k, p.seed, (uint32_t)i, variant, tau, p.Q, p.ldq, p.R,
                     p.ldr, p.perm, p.rank, ws, slice, p.dev_status, d->s[s]);
  }
  for (int s = 0; s < ns; ++s) {
    if (cudaEventRecord(d->join[s], d->s[s]) != cudaSuccess) return RCQR_ECUDA;
    if (cudaStreamWaitEvent(stream, d->join[s], 0) != cudaSuccess) return RCQR_ECUDA;
  }
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
  return (size_t)std::min(count, kMaxStreams) * slice_bytes(probs, count, variant, prec) + 256;
}

rcqr_status rcqr_factor_batched(const rcqr_problem *probs, int count, int variant, int prec, double tau,
                                void *workspace, size_t ws_bytes, cudaStream_t stream) {
  if (!probs || count < 1 || variant < 0 || variant > 3 || !(prec >= 0 && prec <= 2)) return RCQR_EINVAL;
  if ((variant == RCQR_RR || variant == RCQR_RR2) && !(tau >= 0.0)) return RCQR_EINVAL;
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
  if (dev >= 0 && dev < 64) g_best_streams[dev] = best;
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
