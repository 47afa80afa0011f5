// Measured ALU peaks of the device (the denominators of the roofline of the
// FP32 and FP64 kernels): fused multiply-add throughput over every SM.
// Not part of the paper's method; a measurement aid of this library.
#include <cuda_runtime.h>

#include "../../include/spg.h"
#include "spg_internal.h"

namespace spg {
namespace {

// Eight independent FMA chains per thread (enough to hide the pipeline
// latency at full occupancy); the result is stored only under a condition
// that never holds, so that the chains are not removed.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T* out, int iters, T m, T c) {
  T a[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) a[q] = (T)(threadIdx.x + q) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = fma(a[q], m, c);
  }
  T s = T(0);
#pragma unroll
  for (int q = 0; q < 8; ++q) s += a[q];
  if (s == (T)-12345.0) out[blockIdx.x] = s;
}

template <typename T>
int probe(cudaStream_t st, double* tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
    return SPG_ECUDA;
  const int blocks = sms * 8, threads = 256;
  const int iters = sizeof(T) == 4 ? 1 << 17 : 1 << 11;
  T* out = nullptr;
  if (cudaMallocAsync(&out, sizeof(T) * blocks, st) != cudaSuccess) return SPG_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  count_launches("k_fma_probe", st);
  k_fma_probe<T><<<blocks, threads, 0, st>>>(out, iters / 8, (T)0.999999, (T)1e-7);  // warm-up
  cudaEventRecord(e0, st);
  count_launches("k_fma_probe", st);
  k_fma_probe<T><<<blocks, threads, 0, st>>>(out, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e1, st);
  const cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, st);
  if (e != cudaSuccess || ms <= 0.f) return SPG_ECUDA;
  const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return SPG_OK;
}

}  // namespace
}  // namespace spg

extern "C" int spg_peak_probe_stream(void* cuda_stream, int32_t kind, double* tflops) {
  if (!tflops || (kind != 0 && kind != 1)) return SPG_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  return kind == 0 ? spg::probe<float>(st, tflops) : spg::probe<double>(st, tflops);
}
