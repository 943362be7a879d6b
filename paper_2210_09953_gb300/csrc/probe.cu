// Throughput probes for the rooflines of the kernels that are bound by arithmetic
// rather than by memory: the Philox4x32-10 generator that realises Theta (Sec. 2),
// FP32 and FP64 fused multiply-adds and 32-bit integer multiply-adds.
//
// Each probe kernel runs a fixed number of independent operation chains per thread
// over a grid of 4 CTAs of 256 threads per SM, with no memory traffic but one
// checksum store per thread (so nothing is optimised away).  rcqr_probe launches one
// of them on the caller's stream and returns the number of operations it performs;
// the caller times the launch with CUDA events (the library does not synchronise).
#include <cuda_runtime.h>

#include "rcqr_internal.h"
#include "theta.cuh"

namespace rcqr {

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) probe_philox_kernel(int iters, uint32_t k0, uint32_t k1,
                                                                      uint32_t *out) {
  uint32_t rk[20];
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    rk[2 * r] = k0 + (uint32_t)r * 0x9E3779B9u;
    rk[2 * r + 1] = k1 + (uint32_t)r * 0xBB67AE85u;
  }
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint4 w = philox4x32_10_keys(make_uint4((uint32_t)it, t, (uint32_t)c, 0u), rk);
      acc ^= w.x ^ w.y ^ w.z ^ w.w;
    }
  }
  out[t] = acc;
}

__global__ void __launch_bounds__(kProbeThreads) probe_ffma_kernel(int iters, float a, float b, float *out) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_dfma_kernel(int iters, double a, double b, double *out) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_imad_kernel(int iters, uint32_t a, uint32_t b, uint32_t *out) {
  uint32_t x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x + (uint32_t)c;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = x[c] * a + b;
  }
  uint32_t s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s ^= x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

}  // namespace rcqr

using namespace rcqr;

extern "C" {

size_t rcqr_probe_scratch_bytes(void) { return (size_t)4 * 1024 * kProbeThreads * sizeof(double); }

int64_t rcqr_probe(int kind, int iters, void *scratch, size_t scratch_bytes, cudaStream_t stream) {
  if (iters < 1 || !scratch) return -1;
  const int grid = 4 * num_sms();
  if ((size_t)grid * kProbeThreads * sizeof(double) > scratch_bytes) return -1;
  const int64_t threads = (int64_t)grid * kProbeThreads;
  switch (kind) {
    case RCQR_PROBE_PHILOX:
      probe_philox_kernel<<<grid, kProbeThreads, 0, stream>>>(iters, 0x5EED0002u, 0u, (uint32_t *)scratch);
      if (cudaGetLastError() != cudaSuccess) return -1;
      return threads * iters * 4;
    case RCQR_PROBE_FFMA:
      probe_ffma_kernel<<<grid, kProbeThreads, 0, stream>>>(iters, 0.999999f, 1e-7f, (float *)scratch);
      if (cudaGetLastError() != cudaSuccess) return -1;
      return threads * iters * kChains;
    case RCQR_PROBE_DFMA:
      probe_dfma_kernel<<<grid, kProbeThreads, 0, stream>>>(iters, 0.9999999999, 1e-12, (double *)scratch);
      if (cudaGetLastError() != cudaSuccess) return -1;
      return threads * iters * kChains;
    case RCQR_PROBE_IMAD:
      probe_imad_kernel<<<grid, kProbeThreads, 0, stream>>>(iters, 1664525u, 1013904223u, (uint32_t *)scratch);
      if (cudaGetLastError() != cudaSuccess) return -1;
      return threads * iters * kChains;
    default:
      return -1;
  }
}

}  // extern "C"
