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
  const double* dev_flops;  // mapped host slot written by the kernel (or null)
};
struct Agg {
  double ms = 0, flops = 0, bytes = 0, aux = 0;
  int64_t launches = 0;
};
std::mutex g_mu;
std::vector<Rec> g_open;            // recorded, not yet folded in
std::vector<cudaEvent_t> g_pool;    // reusable events
std::map<std::string, Agg> g_agg;
double* g_mapped = nullptr;   // pinned, device-mapped slots for device-computed work
double* g_mapped_dev = nullptr;
int g_mapped_next = 0;
constexpr int MAPPED_SLOTS = 8192;  // pairs of doubles: work, auxiliary count

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
    a.flops += r.flops + (r.dev_flops ? ((volatile const double*)r.dev_flops)[0] : 0.0);
    a.aux += r.dev_flops ? ((volatile const double*)r.dev_flops)[1] : 0.0;
    a.bytes += r.bytes;
    a.launches += 1;
    g_pool.push_back(r.start);
    g_pool.push_back(r.stop);
  }
  g_open.clear();
}
}  // namespace

ProfScope::ProfScope(const char* name, cudaStream_t st, double flops, double bytes, const double* dev_flops_host)
    : s(st) {
  if (!g_prof_on) return;
  std::lock_guard<std::mutex> g(g_mu);
  if (g_open.size() > 4096) fold();
  Rec r{name, get_event(), get_event(), flops, bytes, dev_flops_host};
  CUDA_TRY(cudaEventRecord(r.start, st));
  g_open.push_back(r);
  slot = (int)g_open.size() - 1;
}

ProfScope::~ProfScope() {
  if (slot < 0) return;
  std::lock_guard<std::mutex> g(g_mu);
  cudaEventRecord(g_open[slot].stop, s);
}

// A slot the device writes a launch's work into (host pointer for the profiler,
// device pointer for the kernel); null when profiling is off.
double* prof_work_slot(double** dev) {
  *dev = nullptr;
  if (!g_prof_on) return nullptr;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_mapped) {
    CUDA_TRY(cudaHostAlloc((void**)&g_mapped, 2 * MAPPED_SLOTS * sizeof(double), cudaHostAllocMapped));
    CUDA_TRY(cudaHostGetDevicePointer((void**)&g_mapped_dev, g_mapped, 0));
  }
  if (g_mapped_next >= MAPPED_SLOTS) {
    fold();
    g_mapped_next = 0;
  }
  const int i = 2 * g_mapped_next++;
  g_mapped[i] = 0.0;
  g_mapped[i + 1] = 0.0;
  *dev = g_mapped_dev + i;
  return g_mapped + i;
}

void prof_enable(bool on) {
  std::lock_guard<std::mutex> g(g_mu);
  fold();
  g_agg.clear();
  g_mapped_next = 0;
  g_prof_on = on;
}

int prof_read(int idx, std::string& name, double& ms, int64_t& launches, double& flops, double& bytes,
              double& aux) {
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
    aux = kv.second.aux;
    return 1;
  }
  return 0;
}

}  // namespace tdvp
