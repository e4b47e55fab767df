// Launch accounting: a process-wide count of kernel launches and, while
// profiling is on, CUDA events recorded on the launching stream around every
// kernel launch, aggregated per kernel name.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace eagpt {

namespace {
std::atomic<int64_t> g_launches{0};
std::atomic<bool> g_profiling{false};
std::mutex g_mu;
struct Rec {
  const char* name;
  cudaEvent_t a, b;
};
std::vector<Rec> g_recs;
}  // namespace

LaunchScope::LaunchScope(cudaStream_t st, const char* name) : st_(st), name_(name), a_(nullptr) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (g_profiling.load(std::memory_order_relaxed)) {
    cudaEventCreate(&a_);
    cudaEventRecord(a_, st_);
  }
}

LaunchScope::~LaunchScope() {
  if (a_) {
    cudaEvent_t b;
    cudaEventCreate(&b);
    cudaEventRecord(b, st_);
    std::lock_guard<std::mutex> g(g_mu);
    g_recs.push_back({name_, a_, b});
  }
}

int64_t launch_count() { return g_launches.load(); }

void profile_begin() {
  std::lock_guard<std::mutex> g(g_mu);
  for (auto& r : g_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_recs.clear();
  g_profiling.store(true);
}

int profile_end(eagpt_kernel_time* out, int capacity) {
  g_profiling.store(false);
  std::lock_guard<std::mutex> g(g_mu);
  std::map<std::string, std::pair<int64_t, double>> agg;
  for (auto& r : g_recs) {
    cudaEventSynchronize(r.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    auto& e = agg[r.name];
    e.first += 1;
    e.second += ms;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_recs.clear();
  int k = 0;
  for (auto& kv : agg) {
    if (k < capacity && out) {
      std::memset(out[k].name, 0, sizeof(out[k].name));
      std::strncpy(out[k].name, kv.first.c_str(), sizeof(out[k].name) - 1);
      out[k].launches = kv.second.first;
      out[k].total_ms = kv.second.second;
    }
    ++k;
  }
  return k;
}

}  // namespace eagpt
