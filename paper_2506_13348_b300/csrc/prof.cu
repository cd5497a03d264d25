// Kernel launch accounting and per-stage CUDA-event timing.
//
// Every launch wrapper reports its kernel count (ts_launch_count).  When
// profiling is on, each pipeline stage records a CUDA event pair on the
// stream it launches on; ts_profile_report resolves them after the work
// finished and aggregates launch counts and device time per stage.
#include <atomic>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.h"
#include "prof.h"
#include "../../include/texsplat.h"

namespace ts {

static std::atomic<long long> g_launches{0};
static std::atomic<bool> g_prof{false};
static std::mutex g_mu;
struct Rec {
  std::string name;
  cudaEvent_t a, b;
};
static std::vector<Rec> g_recs;
static std::vector<cudaEvent_t> g_free_events;

void note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static cudaEvent_t get_event() {
  if (!g_free_events.empty()) {
    cudaEvent_t e = g_free_events.back();
    g_free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

ProfScope::ProfScope(cudaStream_t st, const char* name) : st_(st), name_(name), a_(nullptr) {
  if (!g_prof.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  a_ = get_event();
  if (a_) cudaEventRecord(a_, st_);
}

ProfScope::~ProfScope() {
  if (!a_) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = get_event();
  if (!b) return;
  cudaEventRecord(b, st_);
  g_recs.push_back(Rec{name_, a_, b});
}

}  // namespace ts

using namespace ts;

extern "C" {

int64_t ts_launch_count(void) { return g_launches.load(); }

ts_status ts_profile_enable(int on) {
  g_prof.store(on != 0);
  return TS_OK;
}

ts_status ts_profile_report(char* buf, size_t buflen) {
  std::lock_guard<std::mutex> lk(g_mu);
  std::map<std::string, std::pair<long long, double>> agg;
  for (Rec& r : g_recs) {
    float ms = 0.f;
    cudaEventSynchronize(r.b);
    cudaEventElapsedTime(&ms, r.a, r.b);
    auto& e = agg[r.name];
    e.first += 1;
    e.second += ms;
    g_free_events.push_back(r.a);
    g_free_events.push_back(r.b);
  }
  g_recs.clear();
  std::string out;
  char line[256];
  for (auto& kv : agg) {
    snprintf(line, sizeof(line), "%s %lld %.6f\n", kv.first.c_str(), kv.second.first, kv.second.second);
    out += line;
  }
  if (buf && buflen > 0) {
    size_t n = out.size() < buflen - 1 ? out.size() : buflen - 1;
    memcpy(buf, out.data(), n);
    buf[n] = 0;
  }
  return TS_OK;
}

}  // extern "C"
