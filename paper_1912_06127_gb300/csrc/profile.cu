// Per-kernel CUDA-event timing for the benchmark's roofline figures.
#include <map>
#include <mutex>
#include <string>

#include "common.h"

namespace tdvp {

bool g_prof_on = false;

namespace {
struct Rec {
  std::string name;
  cudaEvent_t start, stop;
  double flops, bytes;
};
struct Agg {
  double ms = 0, flops = 0, bytes = 0;
  int64_t launches = 0;
};
std::mutex g_mu;
std::vector<Rec> g_open;            // recorded, not yet folded in
std::vector<cudaEvent_t> g_pool;    // reusable events
std::map<std::string, Agg> g_agg;

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  CUDA_TRY(cudaEventCreate(&e));
  return e;
}

void fold() {
  for (auto& r : g_open) {
    CUDA_TRY(cudaEventSynchronize(r.stop));
    float ms = 0;
    CUDA_TRY(cudaEventElapsedTime(&ms, r.start, r.stop));
    Agg& a = g_agg[r.name];
    a.ms += ms;
    a.flops += r.flops;
    a.bytes += r.bytes;
    a.launches += 1;
    g_pool.push_back(r.start);
    g_pool.push_back(r.stop);
  }
  g_open.clear();
}
}  // namespace

ProfScope::ProfScope(const char* name, cudaStream_t st, double flops, double bytes) : s(st) {
  if (!g_prof_on) return;
  std::lock_guard<std::mutex> g(g_mu);
  if (g_open.size() > 4096) fold();
  Rec r{name, get_event(), get_event(), flops, bytes};
  CUDA_TRY(cudaEventRecord(r.start, st));
  g_open.push_back(r);
  slot = (int)g_open.size() - 1;
}

ProfScope::~ProfScope() {
  if (slot < 0) return;
  std::lock_guard<std::mutex> g(g_mu);
  cudaEventRecord(g_open[slot].stop, s);
}

void prof_enable(bool on) {
  std::lock_guard<std::mutex> g(g_mu);
  fold();
  g_agg.clear();
  g_prof_on = on;
}

int prof_read(int idx, std::string& name, double& ms, int64_t& launches, double& flops, double& bytes) {
  std::lock_guard<std::mutex> g(g_mu);
  fold();
  if (idx < 0) return (int)g_agg.size();
  int i = 0;
  for (auto& kv : g_agg) {
    if (i++ != idx) continue;
    name = kv.first;
    ms = kv.second.ms;
    launches = kv.second.launches;
    flops = kv.second.flops;
    bytes = kv.second.bytes;
    return 1;
  }
  return 0;
}

}  // namespace tdvp
