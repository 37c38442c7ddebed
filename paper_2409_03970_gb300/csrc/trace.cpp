// Kernel tracing: when enabled, every kernel launch of the library is
// bracketed by two CUDA events recorded on the launch's own stream, so that
// per-kernel device durations can be read back without a profiler.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "nsort.h"
#include "nsort_internal.h"

namespace nsort {

namespace {

const char *const kKernelNames[] = {"tile_sort_keys", "tile_sort_pairs", "partition",
                                    "merge_keys",     "merge_pairs",     "segmented_bin",
                                    "segmented_sort", "segmented_merge", "segmented_copy",
                                    "tile_sort_keys64", "merge_keys64",
                                    "sample_merge",   "merge4_bounds",   "merge4_keys"};
constexpr int kNumKernels = sizeof(kKernelNames) / sizeof(kKernelNames[0]);

struct Rec {
  int kernel;
  cudaEvent_t start, stop;
};

std::mutex g_mu;
bool g_enabled = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

}  // namespace

TraceScope::TraceScope(int kernel, cudaStream_t st) : kernel_(kernel), st_(st) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_enabled || kernel < 0 || kernel >= kNumKernels) return;
  start_ = take_event();
  stop_ = take_event();
  if (!start_ || !stop_) return;
  cudaEventRecord(start_, st_);
  active_ = true;
}

TraceScope::~TraceScope() {
  if (!active_) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEventRecord(stop_, st_);
  g_recs.push_back({kernel_, start_, stop_});
}

}  // namespace nsort

using namespace nsort;

extern "C" int nsort_trace_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_enabled = on != 0;
  for (auto &r : g_recs) {
    g_pool.push_back(r.start);
    g_pool.push_back(r.stop);
  }
  g_recs.clear();
  return NSORT_OK;
}

extern "C" int nsort_trace_read(nsort_trace_entry *out, int capacity, int *count) {
  std::lock_guard<std::mutex> lk(g_mu);
  double ms[kNumKernels] = {0};
  uint64_t launches[kNumKernels] = {0};
  int rc = NSORT_OK;
  for (auto &r : g_recs) {
    float t = 0.f;
    if (cudaEventSynchronize(r.stop) != cudaSuccess ||
        cudaEventElapsedTime(&t, r.start, r.stop) != cudaSuccess) {
      set_last_error(std::string("trace: ") + cudaGetErrorString(cudaGetLastError()));
      rc = NSORT_ECUDA;
    }
    ms[r.kernel] += t;
    launches[r.kernel] += 1;
    g_pool.push_back(r.start);
    g_pool.push_back(r.stop);
  }
  g_recs.clear();
  int k = 0;
  for (int i = 0; i < kNumKernels; ++i) {
    if (!launches[i]) continue;
    if (out && k < capacity) {
      std::memset(&out[k], 0, sizeof(out[k]));
      std::strncpy(out[k].kernel, kKernelNames[i], sizeof(out[k].kernel) - 1);
      out[k].launches = launches[i];
      out[k].total_ms = ms[i];
    }
    ++k;
  }
  if (count) *count = k;
  return rc;
}
