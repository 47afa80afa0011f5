// Autotuner of tile shapes.
//
// Several kernels of the path come in variants that differ only in how their
// outputs are spread over threads and blocks -- the SIMT product's outputs per
// thread, the per-state products' states per block, whether the mixed
// marginals stage the boundary-MPS site in shared memory -- while every
// output is computed by the same sequence of operations.  Their results are
// therefore bit-identical, and the fastest one may be used anywhere.  At the
// first launch of a shape (kernel, sizes, strides, instances of the lockstep
// group, device) on a stream that is not being captured, every valid variant
// is run on the real operands and timed with CUDA events on that stream
// (best of three runs each); that launch and every later one of the shape,
// captured into a graph or not, uses the fastest.  A shape first met inside
// a capture, or while the per-kernel profiler records, keeps the built-in
// choice until an uncaptured launch times it.  The variants' extra runs are
// not counted as launches of the library.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>

#include "spg.h"
#include "spg_internal.h"

namespace spg {
namespace {

struct TuneEntry {
  int choice = -1;  // -1: being timed by another host thread
  int n_var = 0;
  float us[TUNE_MAX_VARIANTS] = {};
};

struct Tuner {
  std::mutex mu;
  std::atomic<int> mode{SPG_TUNE_ON};
  std::map<std::string, TuneEntry> cache;
};

Tuner& tuner() {
  static Tuner t;
  return t;
}

int forced_variant(int mode, int n_var, unsigned valid, int dflt) {
  int k = std::min(mode - SPG_TUNE_FORCE, n_var - 1);
  while (k > 0 && !((valid >> k) & 1u)) --k;
  return ((valid >> k) & 1u) ? k : dflt;
}

}  // namespace

int tune_pick(const char* kernel, const long long* shape, int n_shape, cudaStream_t st, int n_var, unsigned valid,
              int dflt, const std::function<void(int)>& launch) {
  Tuner& T = tuner();
  const int mode = T.mode.load();
  n_var = std::min(n_var, TUNE_MAX_VARIANTS);
  valid &= (1u << n_var) - 1u;
  if (mode == SPG_TUNE_OFF || valid == 0) return dflt;
  if (mode >= SPG_TUNE_FORCE) return forced_variant(mode, n_var, valid, dflt);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return dflt;
  std::string key = kernel;
  key += " dev " + std::to_string(dev) + " group " + std::to_string(zn()) + " shape";
  for (int i = 0; i < n_shape; ++i) key += " " + std::to_string(shape[i]);
  {
    std::lock_guard<std::mutex> lock(T.mu);
    auto it = T.cache.find(key);
    if (it != T.cache.end()) return it->second.choice >= 0 ? it->second.choice : dflt;
  }
  // time only outside captures and profiled stretches, and only with no
  // error pending from earlier work (the variants' launch checks would
  // consume it)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return dflt;
  if (kernel_profile().on || cudaPeekAtLastError() != cudaSuccess) return dflt;
  {
    std::lock_guard<std::mutex> lock(T.mu);
    auto r = T.cache.emplace(key, TuneEntry{});
    if (!r.second) return r.first->second.choice >= 0 ? r.first->second.choice : dflt;
  }
  TuneEntry e;
  e.n_var = n_var;
  for (int v = 0; v < TUNE_MAX_VARIANTS; ++v) e.us[v] = -1.f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool ok = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  for (int rep = 0; ok && rep < 3; ++rep)
    for (int v = 0; ok && v < n_var; ++v) {
      if (!((valid >> v) & 1u)) continue;
      if (cudaEventRecord(e0, st) != cudaSuccess) {
        ok = false;
        break;
      }
      launch(v);
      if (cudaGetLastError() != cudaSuccess) {  // a configuration this device refuses
        valid &= ~(1u << v);
        e.us[v] = -1.f;
        continue;
      }
      float ms = 0.f;
      if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        ok = false;
        break;
      }
      const float us = 1e3f * ms;
      if (e.us[v] < 0.f || us < e.us[v]) e.us[v] = us;
    }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  int best = dflt;
  if (ok) {
    float bt = INFINITY;
    for (int v = 0; v < n_var; ++v)
      if (((valid >> v) & 1u) && e.us[v] >= 0.f && e.us[v] < bt) {
        bt = e.us[v];
        best = v;
      }
  } else {
    cudaGetLastError();
  }
  e.choice = best;
  std::lock_guard<std::mutex> lock(T.mu);
  T.cache[key] = e;
  return best;
}

}  // namespace spg

using namespace spg;

extern "C" int spg_autotune_set(int32_t mode, int32_t* previous) {
  if (mode < 0 || mode >= SPG_TUNE_FORCE + TUNE_MAX_VARIANTS) return SPG_EINVAL;
  const int old = tuner().mode.exchange(mode);
  if (previous) *previous = old;
  return SPG_OK;
}

extern "C" int spg_autotune_clear(void) {
  Tuner& T = tuner();
  std::lock_guard<std::mutex> lock(T.mu);
  for (const auto& kv : T.cache)
    if (kv.second.choice < 0) return SPG_EINVAL;  // a shape is being timed
  T.cache.clear();
  return SPG_OK;
}

extern "C" int spg_autotune_report(int32_t* n_shapes, char* text_out, size_t cap) {
  Tuner& T = tuner();
  std::string out;
  int n = 0;
  {
    std::lock_guard<std::mutex> lock(T.mu);
    for (const auto& kv : T.cache) {
      if (kv.second.choice < 0) continue;
      ++n;
      out += kv.first + " -> " + std::to_string(kv.second.choice) + " us";
      for (int v = 0; v < kv.second.n_var; ++v) {
        char b[32];
        std::snprintf(b, sizeof(b), " %.2f", kv.second.us[v]);
        out += b;
      }
      out += "\n";
    }
  }
  if (n_shapes) *n_shapes = n;
  if (text_out && cap > 0) {
    std::strncpy(text_out, out.c_str(), cap - 1);
    text_out[cap - 1] = 0;
  }
  return SPG_OK;
}
