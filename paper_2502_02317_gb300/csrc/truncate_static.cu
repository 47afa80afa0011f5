// spg_truncate_static: the zipper's truncated SVD (the same kernels as
// spg_truncate) for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: an application whose device memory is
// entirely owned by its own pool allocator (a framework's caching allocator,
// or a fixed arena reserved at start-up) leaves nothing for a library to
// allocate and may forbid raw allocations outright; a latency-critical loop
// cannot pay the implicit device synchronisation an allocation may cause;
// and a plug-in that runs after its host application's initialisation
// phase is often not allowed to grow the process's device footprint.  For
// them this entry point takes its scratch from one fixed array compiled into
// the library, so it allocates nothing at call time.
//
// The array below is part of the library image: every GPU on which the
// library is loaded holds it (SPG_TRUNC_STATIC_SCRATCH_BYTES) until the
// process exits.
#include <mutex>

#include "../../include/spg.h"
#include "spg_internal.h"

namespace spg {

// Scratch of the largest call the limits allow (m, n <= 256, keep <= 32):
// the truncation's work buffer plus its sigma_1 and flag words.
constexpr size_t kStaticScratchDoubles = SPG_TRUNC_STATIC_SCRATCH_BYTES / sizeof(double);
static __device__ __align__(256) double g_trunc_scratch[kStaticScratchDoubles];

namespace {

constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_setup_mutex;

// Device address of g_trunc_scratch on the current device.  In host code the
// symbol's name is only a host-side stand-in, so the address is looked up
// once per device (that device current) and cached.
int scratch_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return SPG_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_trunc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return SPG_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return SPG_OK;
}

}  // namespace
}  // namespace spg

using namespace spg;

extern "C" int spg_truncate_static(const double* M, int32_t m, int32_t n, int32_t keep, int32_t iters, double* V,
                                   double* US, double* sigma, void* cuda_stream) {
  if (!M || !V || !US || !sigma) return SPG_EINVAL;
  if (m < 1 || n < 1 || keep < 1 || keep > m || keep > n || iters < 0 || iters > 64) return SPG_EINVAL;
  if (m > SPG_TRUNC_STATIC_MAX_DIM || n > SPG_TRUNC_STATIC_MAX_DIM || keep > SPG_TRUNC_STATIC_MAX_KEEP)
    return SPG_EUNSUPPORTED;  // beyond the static scratch
  const size_t work = truncated_svd_work(m, n, keep);
  if (work + 8 > kStaticScratchDoubles) return SPG_EUNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // the call waits for its stream before returning, which a stream under
  // capture does not allow (the wait would invalidate the caller's capture):
  // such a stream is rejected before anything is enqueued on it
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return SPG_ECUDA;
  }
  if (cs != cudaStreamCaptureStatusNone) return SPG_EINVAL;
  double* base = nullptr;
  const int rc = scratch_address(&base);
  if (rc != SPG_OK) return rc;
  double* s1 = base + work;
  int* flag = reinterpret_cast<int*>(base + work + 2);
  // the degenerate-cut counter must start at zero; every other word of the
  // scratch is written by the kernels before it is read
  if (cudaMemsetAsync(flag, 0, sizeof(int) * 2, st) != cudaSuccess) return SPG_ECUDA;
  if (truncated_svd<double>(M, m, n, keep, iters, 0x5eedull, V, US, base, work, s1, flag, st) != cudaSuccess)
    return SPG_ECUDA;
  if (cudaMemcpyAsync(sigma, base + truncated_svd_sigma_offset(m, n, keep), sizeof(double) * keep,
                      cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return SPG_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SPG_ECUDA;
  return SPG_OK;
}
