// rcqr_sketch_noalloc: the sketch P = Theta X without a caller workspace.
//
// Some callers cannot hand the library scratch memory: a plugin whose fixed
// argument list has no slot for a workspace pointer, or code running inside a
// host application whose device memory is owned entirely by that
// application's pool, where an extra cudaMalloc is forbidden or would fail.
// For them the per-CTA partial sums of the sketch live in one file-scope
// device array, g_sketch_scratch, of kScratchDoubles doubles (8 MiB).  Every
// GPU that loads the library keeps that array until the process exits.
//
// The device address of the array is looked up once per device, on the first
// call made with that device current (cudaGetSymbolAddress); that first call
// on each device should therefore come before any stream capture.  All calls
// share the one array and it keeps the last call's contents: two calls whose
// work overlaps on the GPU (different streams without ordering between them)
// race on it.  Nothing in the array needs to start at zero: each call writes
// every partial it later reads.
#include <cuda_runtime.h>

#include <mutex>

#include "rcqr_internal.h"

namespace {

constexpr size_t kScratchDoubles = size_t(1) << 20;  // 8 MiB

__device__ __align__(256) double g_sketch_scratch[kScratchDoubles];

std::mutex g_mu;
double *g_scratch_ptr[64] = {nullptr};

// Device address of g_sketch_scratch for the current device (set-up on first use).
cudaError_t scratch_for_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sketch_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" rcqr_status rcqr_sketch_noalloc(const void *X, int64_t m, int64_t n, int64_t ldx,
                                           int prec, int64_t k, uint64_t seed, int64_t row_offset,
                                           double *P, int64_t ldp, double *colnorm2,
                                           cudaStream_t stream) {
  if (!X || !P || !(prec == RCQR_F64 || prec == RCQR_F32 || prec == RCQR_BF16) || m < 1 || n < 1 ||
      n > 256 || k < n || k > 2048 || (k % 8) != 0 || ldx < m || ldp < k || row_offset < 0)
    return RCQR_EINVAL;
  // one row group needs n*k doubles, the column norms 2*SMs*n more
  const size_t need = (size_t)n * k + (colnorm2 ? (size_t)2 * rcqr::num_sms() * n : 0);
  if (need > kScratchDoubles) return RCQR_EWORKSPACE;
  double *scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return RCQR_ECUDA;
  const cudaError_t e = rcqr::launch_sketch_into(X, m, n, ldx, prec, k, seed, row_offset, P, ldp,
                                                 colnorm2, scratch, kScratchDoubles, stream);
  if (e == cudaErrorInvalidValue) return RCQR_EWORKSPACE;
  return e == cudaSuccess ? RCQR_OK : RCQR_ECUDA;
}
