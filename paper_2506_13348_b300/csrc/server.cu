// Continuous-batching view server (host runtime, C++).
//
// Requests (scene, camera) are queued by ts_server_submit and return a
// ticket at once.  Each worker thread owns a non-blocking CUDA stream; when
// it is free it takes every queued request that fits -- up to max_batch
// views, same atlas dtype, and within the device-memory budget -- and
// renders them with one ts_render_views launch sequence.  Requests that
// arrive while batches are on the GPU join the next batch a worker forms,
// and batches of different workers overlap on the device.  Latency is taken
// from submission to the completion of the batch's last kernel.  Results
// stay on the device until ts_server_wait copies them out.
//
// Memory admission: a request is admitted against the budget with its
// output, the exact per-splat buffers of the render, and an estimate of its
// pair buffers (pairs per pixel, learned per scene as the largest value seen,
// 32 before the first render).  Once a batch has counted its pairs (the
// render's one synchronisation) the reservation is trued up to the exact
// bytes still to be allocated: a surplus is returned at once; a deficit
// waits until running batches free enough, unless every running batch is
// waiting too (then it proceeds and is counted as over budget, since waiting
// could not end).  A batch whose own memory exceeds the budget fails with
// TS_ERR_CAPACITY, and so does a queued request once its scene's learned
// pair count puts it above the whole budget.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kernels.h"
#include "../../include/texsplat.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

struct Request {
  uint64_t id = 0;
  ts_scene* scene = nullptr;
  ts_camera cam;
  int dtype = 0;
  size_t out_bytes = 0;
  size_t fixed = 0;  // exact per-splat render buffers
  size_t pairs = 0;  // estimated pair buffers
  size_t cost = 0;   // admission bytes: output + fixed + pairs
  float* out = nullptr;
  double t_submit = 0.0, t_done = 0.0;
  int state = 0;     // 0 queued, 1 running, 2 done, 3 failed
  bool admitted = false;  // its cost was added to the server's reserved bytes
  ts_status status = TS_OK;
  std::string err;
};

}  // namespace

struct ts_server {
  int device = 0;
  size_t arena = 0;
  size_t inflight = 0;
  int max_batch = 8;
  bool stop = false;
  uint64_t next_id = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> reqs;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  cudaStream_t copy_stream = nullptr;
  // admission: batches between admission and completion, those waiting in
  // their true-up, pairs per pixel seen per scene
  int running = 0, waiting = 0;
  std::unordered_map<const ts_scene*, double> ppp;
  cudaEvent_t ref_event = nullptr;  // time origin of the batch log
  // statistics
  std::vector<double> lat_ms;
  int64_t submitted = 0, completed = 0, rejected = 0, failed = 0, batches = 0, batched_views = 0;
  int64_t true_ups = 0, over_budget = 0;
  size_t peak_reserved = 0;
  double pixels = 0.0, t_first = 0.0, t_last = 0.0;
  struct BatchRec {
    int worker, views;
    double t0_ms, t1_ms;
  };
  std::vector<BatchRec> log;  // the last kLogMax batches, oldest first
};

namespace {

constexpr double kInitialPairsPerPixel = 32.0;
constexpr size_t kLogMax = 4096;

// Pair buffers of a view (4 x 4 B per pair, tile ranges and launch orders)
// for `ppp` pairs per pixel.
size_t pair_estimate(const ts_camera& c, double ppp) {
  const size_t px = (size_t)c.width * c.height;
  const size_t tiles = (size_t)((c.width + 15) / 16) * ((c.height + 15) / 16);
  return (size_t)(ppp * (double)px) * 16 + tiles * 24 + 4096;
}

void note_inflight(ts_server* sv) { sv->peak_reserved = std::max(sv->peak_reserved, sv->inflight); }

// A request's admission bytes under the pairs per pixel its scene has shown
// so far (at least the initial estimate).  Caller holds sv->mu.
void refresh_cost(ts_server* sv, Request* r) {
  auto it = sv->ppp.find(r->scene);
  r->pairs = pair_estimate(r->cam, std::max(kInitialPairsPerPixel, it == sv->ppp.end() ? 0.0 : it->second));
  r->cost = r->out_bytes + r->fixed + r->pairs;
}

// True-up of a batch's reservation once its pair count is known (called by
// the render between its synchronisation and its pair-buffer allocations).
struct TrueUp {
  ts_server* sv;
  size_t reserved_pairs;   // the batch's pair estimate, reserved at admission
  size_t reserved_fixed;   // its exact per-splat bytes
  size_t held = 0;         // what the batch holds after the true-up (fixed + pairs)
  double batch_px = 0.0;
  std::vector<ts_scene*> scenes;
};

int true_up(void* ctx, size_t bytes, long long pairs) {
  TrueUp* tu = static_cast<TrueUp*>(ctx);
  ts_server* sv = tu->sv;
  std::unique_lock<std::mutex> lk(sv->mu);
  const double seen = tu->batch_px > 0 ? (double)pairs / tu->batch_px : 0.0;
  for (ts_scene* s : tu->scenes) {
    auto it = sv->ppp.find(s);
    if (it == sv->ppp.end() || it->second < seen) sv->ppp[s] = seen;
  }
  if (tu->reserved_fixed + bytes > sv->arena) {
    sv->inflight -= tu->reserved_pairs;
    tu->reserved_pairs = 0;
    tu->held = tu->reserved_fixed;
    sv->cv_work.notify_all();
    return ts::set_error(TS_ERR_CAPACITY, "server: the batch's pair buffers exceed the memory budget");
  }
  if (bytes <= tu->reserved_pairs) {
    sv->inflight -= tu->reserved_pairs - bytes;
    sv->cv_work.notify_all();
  } else {
    const size_t extra = bytes - tu->reserved_pairs;
    ++sv->true_ups;
    ++sv->waiting;
    while (sv->inflight + extra > sv->arena) {
      if (sv->waiting >= sv->running) {  // every running batch waits: none will free memory
        ++sv->over_budget;
        break;
      }
      sv->cv_work.wait(lk);
    }
    --sv->waiting;
    sv->inflight += extra;
    note_inflight(sv);
  }
  tu->held = tu->reserved_fixed + bytes;
  return TS_OK;
}

void worker_loop(ts_server* sv, int w) {
  cudaSetDevice(sv->device);
  cudaStream_t st = sv->streams[w];
  cudaEvent_t ev, ev0;
  cudaEventCreateWithFlags(&ev, cudaEventBlockingSync);
  cudaEventCreate(&ev0);
  std::vector<Request*> batch;
  std::vector<ts_scene*> scenes;
  std::vector<ts_camera> cams;
  std::vector<float*> outs;
  for (;;) {
    batch.clear();
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      // wake for a front request that fits, or that no longer can fit
      sv->cv_work.wait(lk, [&] {
        if (sv->stop) return true;
        if (sv->queue.empty()) return false;
        refresh_cost(sv, sv->queue.front());
        return sv->queue.front()->cost > sv->arena || sv->inflight + sv->queue.front()->cost <= sv->arena;
      });
      if (sv->stop) break;
      // requests that their scene's learned pair count puts above the whole
      // budget (admitted to the queue on a smaller estimate) fail here
      // instead of blocking the queue
      bool failed_any = false;
      while (!sv->queue.empty()) {
        Request* r = sv->queue.front();
        refresh_cost(sv, r);
        if (r->cost <= sv->arena) break;
        sv->queue.pop_front();
        r->state = 3;
        r->status = TS_ERR_CAPACITY;
        r->err = "server: the scene's pair count puts the request above the memory budget";
        r->t_done = now_s();
        ++sv->failed;
        failed_any = true;
      }
      if (failed_any) sv->cv_done.notify_all();
      if (sv->queue.empty()) continue;
      const int dtype = sv->queue.front()->dtype;
      while (!sv->queue.empty() && (int)batch.size() < sv->max_batch) {
        Request* r = sv->queue.front();
        if (r->dtype != dtype) break;
        refresh_cost(sv, r);  // the pair estimate from what this scene's renders have shown so far
        if (sv->inflight + r->cost > sv->arena) break;
        sv->queue.pop_front();
        sv->inflight += r->cost;
        r->state = 1;
        r->admitted = true;
        batch.push_back(r);
      }
      if (!batch.empty()) {
        ++sv->running;
        note_inflight(sv);
      }
    }
    if (batch.empty()) continue;
    TrueUp tu;
    tu.sv = sv;
    tu.reserved_pairs = 0;
    tu.reserved_fixed = 0;
    for (Request* r : batch) {
      tu.reserved_pairs += r->pairs;
      tu.reserved_fixed += r->fixed;
      tu.batch_px += (double)r->cam.width * r->cam.height;
      tu.scenes.push_back(r->scene);
    }
    tu.held = tu.reserved_fixed + tu.reserved_pairs;
    scenes.clear();
    cams.clear();
    outs.clear();
    ts_status st_all = TS_OK;
    std::string err;
    for (Request* r : batch) {
      if (cudaMallocAsync((void**)&r->out, r->out_bytes, st) != cudaSuccess) {
        r->out = nullptr;
        st_all = TS_ERR_OOM;
        err = "server: output allocation failed";
        break;
      }
      scenes.push_back(r->scene);
      cams.push_back(r->cam);
      outs.push_back(r->out);
    }
    cudaEventRecord(ev0, st);
    if (st_all == TS_OK) {
      st_all = ts::render_views_hooked(scenes.data(), cams.data(), (int)batch.size(), outs.data(), nullptr, st,
                                       true_up, &tu);
      if (st_all != TS_OK) err = ts_last_error();
    }
    if (st_all == TS_OK && (cudaEventRecord(ev, st) != cudaSuccess || cudaEventSynchronize(ev) != cudaSuccess)) {
      st_all = TS_ERR_CUDA;
      err = "server: batch completion wait failed";
    }
    float t0_ms = 0.f, t1_ms = 0.f;
    const bool timed = st_all == TS_OK && cudaEventElapsedTime(&t0_ms, sv->ref_event, ev0) == cudaSuccess &&
                       cudaEventElapsedTime(&t1_ms, sv->ref_event, ev) == cudaSuccess;
    const double t = now_s();
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      ++sv->batches;
      sv->batched_views += (int64_t)batch.size();
      --sv->running;
      sv->inflight -= tu.held;  // the batch's render memory; the outputs stay until collected
      if (timed) {
        if (sv->log.size() >= kLogMax) sv->log.erase(sv->log.begin());
        sv->log.push_back({w, (int)batch.size(), (double)t0_ms, (double)t1_ms});
      }
      for (Request* r : batch) {
        r->t_done = t;
        r->status = st_all;
        r->err = err;
        r->state = st_all == TS_OK ? 2 : 3;
        if (st_all == TS_OK) {
          ++sv->completed;
          sv->lat_ms.push_back(1e3 * (r->t_done - r->t_submit));
          sv->pixels += (double)r->cam.width * r->cam.height;
          sv->t_last = std::max(sv->t_last, t);
        } else {
          ++sv->failed;
        }
      }
    }
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
  }
  cudaEventDestroy(ev);
  cudaEventDestroy(ev0);
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (double)(v.size() - 1);
  const size_t i = (size_t)pos;
  const double f = pos - (double)i;
  return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

ts_status ts_server_create(ts_server** out, int device, size_t arena_bytes, int n_streams, int max_batch) {
  if (!out) return ts::set_error(TS_ERR_ARG, "ts_server_create: out is NULL");
  if (n_streams < 1 || n_streams > 16) return ts::set_error(TS_ERR_ARG, "ts_server_create: n_streams in [1, 16]");
  if (max_batch < 1 || max_batch > 32) return ts::set_error(TS_ERR_ARG, "ts_server_create: max_batch in [1, 32]");
  if (arena_bytes == 0) return ts::set_error(TS_ERR_ARG, "ts_server_create: arena_bytes must be > 0");
  if (cudaSetDevice(device) != cudaSuccess) return ts::set_error(TS_ERR_ARG, "ts_server_create: bad device");
  ts_server* sv = new (std::nothrow) ts_server();
  if (!sv) return ts::set_error(TS_ERR_OOM, "ts_server_create: host allocation failed");
  sv->device = device;
  sv->arena = arena_bytes;
  sv->max_batch = max_batch;
  sv->streams.resize(n_streams);
  for (int i = 0; i < n_streams; ++i) {
    if (cudaStreamCreateWithFlags(&sv->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
      for (int j = 0; j < i; ++j) cudaStreamDestroy(sv->streams[j]);
      delete sv;
      return ts::set_error(TS_ERR_CUDA, "ts_server_create: stream creation failed");
    }
  }
  cudaStreamCreateWithFlags(&sv->copy_stream, cudaStreamNonBlocking);
  if (cudaEventCreate(&sv->ref_event) != cudaSuccess || cudaEventRecord(sv->ref_event, sv->streams[0]) != cudaSuccess ||
      cudaEventSynchronize(sv->ref_event) != cudaSuccess) {
    for (cudaStream_t s : sv->streams) cudaStreamDestroy(s);
    if (sv->copy_stream) cudaStreamDestroy(sv->copy_stream);
    delete sv;
    return ts::set_error(TS_ERR_CUDA, "ts_server_create: event creation failed");
  }
  for (int i = 0; i < n_streams; ++i) sv->workers.emplace_back(worker_loop, sv, i);
  *out = sv;
  return TS_OK;
}

ts_status ts_server_destroy(ts_server* sv) {
  if (!sv) return TS_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  for (std::thread& t : sv->workers) t.join();
  cudaSetDevice(sv->device);
  cudaDeviceSynchronize();
  for (auto& kv : sv->reqs) {
    if (kv.second->out) cudaFree(kv.second->out);
    delete kv.second;
  }
  for (cudaStream_t s : sv->streams) cudaStreamDestroy(s);
  if (sv->copy_stream) cudaStreamDestroy(sv->copy_stream);
  if (sv->ref_event) cudaEventDestroy(sv->ref_event);
  delete sv;
  return TS_OK;
}

ts_status ts_server_submit(ts_server* sv, ts_scene* scene, const ts_camera* cam, uint64_t* ticket) {
  if (!sv || !scene || !cam || !ticket) return ts::set_error(TS_ERR_ARG, "ts_server_submit: NULL argument");
  if (cam->width < 1 || cam->height < 1 || cam->width > 16384 || cam->height > 16384)
    return ts::set_error(TS_ERR_ARG, "ts_server_submit: bad resolution");
  int64_t n = 0;
  int dtype = 0;
  ts_status q = ts_scene_info(scene, &n, nullptr, &dtype);
  if (q != TS_OK) return q;
  Request* r = new (std::nothrow) Request();
  if (!r) return ts::set_error(TS_ERR_OOM, "ts_server_submit: host allocation failed");
  r->scene = scene;
  r->cam = *cam;
  r->dtype = dtype;
  r->out_bytes = (size_t)cam->width * cam->height * 16;
  r->fixed = ts::render_views_fixed_bytes(n);
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    refresh_cost(sv, r);
    if (r->cost > sv->arena) {
      ++sv->rejected;
      delete r;
      return ts::set_error(TS_ERR_CAPACITY, "ts_server_submit: request larger than the server's memory budget");
    }
    r->id = sv->next_id++;
    if (sv->submitted == 0) sv->t_first = r->t_submit;
    ++sv->submitted;
    sv->reqs[r->id] = r;
    sv->queue.push_back(r);
    *ticket = r->id;
  }
  sv->cv_work.notify_one();
  return TS_OK;
}

ts_status ts_server_wait(ts_server* sv, uint64_t ticket, float* out_rgba, int out_on_device, double timeout_s) {
  if (!sv) return ts::set_error(TS_ERR_ARG, "ts_server_wait: NULL server");
  Request* r = nullptr;
  {
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return ts::set_error(TS_ERR_ARG, "ts_server_wait: unknown ticket");
    r = it->second;
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0));
    while (r->state < 2) {
      if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->state < 2)
        return ts::set_error(TS_ERR_TIMEOUT, "ts_server_wait: timed out");
    }
    sv->reqs.erase(ticket);
  }
  ts_status st = r->status;
  std::string err = r->err;
  if (st == TS_OK && out_rgba) {
    cudaSetDevice(sv->device);
    cudaError_t e = cudaMemcpyAsync(out_rgba, r->out, r->out_bytes,
                                    out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    sv->copy_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sv->copy_stream);
    if (e != cudaSuccess) {
      st = TS_ERR_CUDA;
      err = std::string("ts_server_wait: copy: ") + cudaGetErrorString(e);
    }
  }
  if (r->out) cudaFreeAsync(r->out, sv->copy_stream);
  if (r->admitted) {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->inflight -= r->out_bytes;
  }
  sv->cv_work.notify_all();
  delete r;
  if (st != TS_OK) return ts::set_error(st, err);
  return TS_OK;
}

ts_status ts_server_stats(ts_server* sv, ts_serve_stats* out) {
  if (!sv || !out) return ts::set_error(TS_ERR_ARG, "ts_server_stats: NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  memset(out, 0, sizeof(*out));
  out->submitted = sv->submitted;
  out->completed = sv->completed;
  out->rejected = sv->rejected;
  out->failed = sv->failed;
  out->batches = sv->batches;
  out->mean_batch = sv->batches ? (double)sv->batched_views / (double)sv->batches : 0.0;
  out->p50_ms = percentile(sv->lat_ms, 0.50);
  out->p99_ms = percentile(sv->lat_ms, 0.99);
  double sum = 0.0;
  for (double v : sv->lat_ms) sum += v;
  out->mean_ms = sv->lat_ms.empty() ? 0.0 : sum / (double)sv->lat_ms.size();
  const double span = sv->t_last - sv->t_first;
  out->fps = span > 0 ? (double)sv->completed / span : 0.0;
  out->mpix_per_s = span > 0 ? sv->pixels / span / 1e6 : 0.0;
  out->true_ups = sv->true_ups;
  out->over_budget = sv->over_budget;
  out->peak_reserved_bytes = (double)sv->peak_reserved;
  return TS_OK;
}

ts_status ts_server_request_bytes(ts_server* sv, ts_scene* scene, const ts_camera* cam, size_t* bytes) {
  if (!sv || !scene || !cam || !bytes) return ts::set_error(TS_ERR_ARG, "ts_server_request_bytes: NULL argument");
  int64_t n = 0;
  ts_status q = ts_scene_info(scene, &n, nullptr, nullptr);
  if (q != TS_OK) return q;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->ppp.find(scene);
  *bytes = (size_t)cam->width * cam->height * 16 + ts::render_views_fixed_bytes(n) +
           pair_estimate(*cam, std::max(kInitialPairsPerPixel, it == sv->ppp.end() ? 0.0 : it->second));
  return TS_OK;
}

ts_status ts_server_batch_log(ts_server* sv, int32_t max_entries, int32_t* n_out, int32_t* worker, int32_t* views,
                              double* t0_ms, double* t1_ms) {
  if (!sv || !n_out || max_entries < 0 || (max_entries > 0 && (!worker || !views || !t0_ms || !t1_ms)))
    return ts::set_error(TS_ERR_ARG, "ts_server_batch_log: bad argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  const size_t n = std::min<size_t>((size_t)max_entries, sv->log.size());
  const size_t first = sv->log.size() - n;
  for (size_t i = 0; i < n; ++i) {
    const auto& b = sv->log[first + i];
    worker[i] = b.worker;
    views[i] = b.views;
    t0_ms[i] = b.t0_ms;
    t1_ms[i] = b.t1_ms;
  }
  *n_out = (int32_t)n;
  return TS_OK;
}

ts_status ts_server_reset_stats(ts_server* sv) {
  if (!sv) return ts::set_error(TS_ERR_ARG, "ts_server_reset_stats: NULL server");
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->lat_ms.clear();
  sv->submitted = sv->completed = sv->rejected = sv->failed = sv->batches = sv->batched_views = 0;
  sv->pixels = 0.0;
  sv->true_ups = sv->over_budget = 0;
  sv->peak_reserved = sv->inflight;
  sv->log.clear();
  // the throughput window starts now (or at the next submission)
  sv->t_first = now_s();
  sv->t_last = 0.0;
  return TS_OK;
}

}  // extern "C"
