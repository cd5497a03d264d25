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

// FP32 FMA-rate probe: eight independent fmaf chains per thread (scalar) or
// four float2 chains (paired), on a grid of 8 CTAs x 256 threads per SM.
// The chains converge to a fixed point, so values stay finite; the final
// store is conditional on a value the chains never reach, which keeps the
// compiler from removing them.
constexpr int FP_THREADS = 256;
constexpr int FP_UNROLL = 16;

__global__ void __launch_bounds__(FP_THREADS) k_fma_scalar(float* out, int iters, float seed) {
  float a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = seed * (float)(threadIdx.x + i);
  const float m = 0.999999f, c = 1e-7f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < FP_UNROLL; ++u) {
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = fmaf(a[i], m, c);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  if (s == -1.0f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(FP_THREADS) k_fma_paired(float* out, int iters, float seed) {
  float2 a[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) a[i] = f2(seed * (float)(threadIdx.x + i), seed * (float)(threadIdx.x + 4 + i));
  const float2 m = f2(0.999999f, 0.999999f), c = f2(1e-7f, 1e-7f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < FP_UNROLL; ++u) {
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = fma2(a[i], m, c);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) s += a[i].x + a[i].y;
  if (s == -1.0f) out[blockIdx.x] = s;
}

extern "C" {

ts_status ts_measure_fp32_peak(int device, double* scalar_tflops, double* paired_tflops) {
  if (!scalar_tflops || !paired_tflops) return TS_ERR_ARG;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return TS_ERR_CUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int grid = sms * 8, iters = 2048;
  const double flops = 2.0 * grid * FP_THREADS * (double)iters * FP_UNROLL * 8;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ts_status st = TS_OK;
  if (cudaMalloc(&out, grid * sizeof(float)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    st = TS_ERR_CUDA;
  } else {
    for (int kind = 0; kind < 2 && st == TS_OK; ++kind) {
      float best = 1e30f;
      for (int rep = 0; rep < 4; ++rep) {  // first run warms up
        cudaEventRecord(e0, 0);
        if (kind == 0)
          k_fma_scalar<<<grid, FP_THREADS>>>(out, iters, 1e-3f);
        else
          k_fma_paired<<<grid, FP_THREADS>>>(out, iters, 1e-3f);
        cudaEventRecord(e1, 0);
        note_launches(1);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          st = TS_ERR_CUDA;
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
      }
      const double tf = flops / (best * 1e-3) / 1e12;
      if (kind == 0)
        *scalar_tflops = tf;
      else
        *paired_tflops = tf;
    }
  }
  if (cudaGetLastError() != cudaSuccess) st = TS_ERR_CUDA;
  if (out) cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaSetDevice(prev);
  return st;
}

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
