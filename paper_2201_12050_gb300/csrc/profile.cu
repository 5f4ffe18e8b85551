// Kernel telemetry (profile.cuh): per-kernel CUDA-event timing on the
// launching stream and a process-wide launch counter.
#include <atomic>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "profile.cuh"

namespace fmpb {

namespace {
std::atomic<uint64_t> g_launches{0};
std::atomic<bool> g_enabled{false};
struct Rec {
  const char* name;
  cudaEvent_t a, b;
};
std::mutex g_mu;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

thread_local const char* t_failed_launch = nullptr;

void note_launch(const char* name) {
  if (!t_failed_launch && cudaPeekAtLastError() != cudaSuccess) t_failed_launch = name;
}

const char* take_failed_launch() {
  const char* n = t_failed_launch;
  t_failed_launch = nullptr;
  return n;
}

bool profiling_enabled() { return g_enabled.load(std::memory_order_relaxed); }
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

ProfScope::ProfScope(const char* name, cudaStream_t st) : name_(name), st_(st), slot_(-1) {
  if (!profiling_enabled()) return;
  std::lock_guard<std::mutex> lk(g_mu);
  Rec r{name, take_event(), take_event()};
  if (!r.a || !r.b) return;
  cudaEventRecord(r.a, st);
  g_recs.push_back(r);
  slot_ = (int)g_recs.size() - 1;
}

ProfScope::~ProfScope() {
  if (slot_ < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (slot_ < (int)g_recs.size()) cudaEventRecord(g_recs[slot_].b, st_);
}

}  // namespace fmpb

using namespace fmpb;

extern "C" {

uint64_t fmpb_kernel_launches(void) { return g_launches.load(); }

void fmpb_profile_enable(int on) { g_enabled.store(on != 0); }

fmpb_status fmpb_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  return FMPB_OK;
}

fmpb_status fmpb_profile_summary(char* buf, size_t len) {
  if (!buf || len < 2) {
    set_error("profile_summary: buffer too small");
    return FMPB_EINVAL;
  }
  std::map<std::string, std::pair<long, double>> agg;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& r : g_recs) {
      if (cudaEventSynchronize(r.b) != cudaSuccess) return cuda_status(cudaGetLastError(), "profile_summary");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, r.a, r.b);
      auto& e = agg[r.name];
      e.first += 1;
      e.second += ms;
    }
  }
  std::string out = "{";
  bool first = true;
  for (auto& kv : agg) {
    char line[256];
    snprintf(line, sizeof(line), "%s\"%s\": [%ld, %.6f]", first ? "" : ", ", kv.first.c_str(), kv.second.first,
             kv.second.second);
    out += line;
    first = false;
  }
  out += "}";
  if (out.size() + 1 > len) {
    set_error("profile_summary: needs %zu bytes", out.size() + 1);
    return FMPB_EINVAL;
  }
  memcpy(buf, out.c_str(), out.size() + 1);
  return FMPB_OK;
}

}  // extern "C"
