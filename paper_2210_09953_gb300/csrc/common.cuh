// Small device helpers shared by the kernels of librcqr.so.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace rcqr {

__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return (double)x; }
__device__ __forceinline__ double to_f64(__nv_bfloat16 x) { return (double)__bfloat162float(x); }

template <class T>
__device__ __forceinline__ T from_f64(double x);
template <>
__device__ __forceinline__ double from_f64<double>(double x) { return x; }
template <>
__device__ __forceinline__ float from_f64<float>(double x) { return __double2float_rn(x); }

// Sum over a block of `nthreads` threads (multiple of 32); `red` has >= 32 slots.
// Every thread gets the total.  Fixed order: deterministic.
__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < nw; ++w) t += red[w];
  return t;
}

// sum_{g < G} src[g * stride] by one warp in a fixed order (lane l adds g = l, l+32, ...
// in increasing order, then a fixed shuffle-down tree); the total is returned in lane 0.
__device__ __forceinline__ double warp_sum_strided(const double *src, int G, int64_t stride) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int g = lane; g < G; g += 32) s += src[(int64_t)g * stride];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  return s;
}

}  // namespace rcqr
