// Online tile autotuner for the GEMM launches.
//
// Every GEMM family (the tcgen05 TF32 products, the FP64 and double-float
// SIMT products) has several tile shapes that compute each output element
// with the same sequence of operations, so they give bitwise the same result
// and differ only in speed: which one is fastest depends on the problem shape
// (chi, the MPO bond dimension m and the local dimension d fix M, N, K) and on
// how many problems a stage batches. The first launch of a family with a new
// shape key runs every candidate on the launch's own operands, timed with CUDA
// events on the launching stream (the output is overwritten each time, so
// nothing accumulates), keeps the fastest and records the decision; later
// launches with that key use it. Keys bucket M, N and K to powers of two, so a
// sweep whose bond dimensions grow meets a bounded number of them.
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "common.h"

namespace tdvp {

namespace {

struct Decision {
  int choice;
  std::vector<float> us;  // per candidate, microseconds
};

std::mutex g_tune_mu;
bool g_tune_on = true;
std::map<std::tuple<int, int, int, int, int, int>, Decision> g_tune;

int bucket(int64_t x) {
  int b = 0;
  while (b < 40 && (int64_t(1) << b) < x) ++b;
  return b;
}

}  // namespace

void tune_enable(bool on) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune_on = on;
  g_tune.clear();
}

bool tune_enabled() {
  std::lock_guard<std::mutex> g(g_tune_mu);
  return g_tune_on;
}

int tune_pick(int family, int64_t M, int64_t N, int64_t K, int n, int n_cand, bool may_repeat,
              const std::function<void(int)>& run, cudaStream_t s) {
  const auto key = std::make_tuple(family, bucket(M), bucket(N), bucket(K), bucket(n), n_cand);
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    if (!g_tune_on || !may_repeat) {
      run(0);
      return 0;
    }
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      run(it->second.choice);
      return it->second.choice;
    }
  }
  // time every candidate once on this launch's operands; the last one run is
  // the chosen one, so its output is the one left behind
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  Decision d;
  d.us.assign(n_cand, 0.f);
  for (int c = 0; c < n_cand; ++c) {
    CUDA_TRY(cudaEventRecord(e0, s));
    run(c);
    CUDA_TRY(cudaEventRecord(e1, s));
    CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    d.us[c] = 1e3f * ms;
  }
  d.choice = 0;
  for (int c = 1; c < n_cand; ++c)
    if (d.us[c] < d.us[d.choice]) d.choice = c;
  if (d.choice != n_cand - 1) run(d.choice);
  CUDA_TRY(cudaEventDestroy(e0));
  CUDA_TRY(cudaEventDestroy(e1));
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune[key] = d;
  return d.choice;
}

std::string tune_report() {
  static const char* fam[] = {"tc_gemm_tf32", "tc_gemm_tf32x3", "zgemm_fp64", "zgemm_dd"};
  static const char* cand[][2] = {{"BN256", "BN128"}, {"BN256", "BN128"}, {"64x64", "32x32"}, {"64x64", "32x32"}};
  std::lock_guard<std::mutex> g(g_tune_mu);
  std::string out = "[";
  bool first = true;
  for (const auto& kv : g_tune) {
    const int f = std::get<0>(kv.first);
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s{\"family\": \"%s\", \"M<=\": %lld, \"N<=\": %lld, \"K<=\": %lld, "
                  "\"batch<=\": %lld, \"choice\": \"%s\", \"us\": [",
                  first ? "" : ", ", (f >= 0 && f < 4) ? fam[f] : "?", 1ll << std::get<1>(kv.first),
                  1ll << std::get<2>(kv.first), 1ll << std::get<3>(kv.first), 1ll << std::get<4>(kv.first),
                  (f >= 0 && f < 4 && kv.second.choice < 2) ? cand[f][kv.second.choice] : "?");
    out += buf;
    for (size_t c = 0; c < kv.second.us.size(); ++c) {
      std::snprintf(buf, sizeof(buf), "%s%.1f", c ? ", " : "", kv.second.us[c]);
      out += buf;
    }
    out += "]}";
    first = false;
  }
  out += "]";
  return out;
}

}  // namespace tdvp
