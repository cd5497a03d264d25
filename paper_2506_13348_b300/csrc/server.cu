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
  size_t cost = 0;   // admission bytes (output + estimated binning memory)
  float* out = nullptr;
  double t_submit = 0.0, t_done = 0.0;
  int state = 0;     // 0 queued, 1 running, 2 done, 3 failed
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
  // statistics
  std::vector<double> lat_ms;
  int64_t submitted = 0, completed = 0, rejected = 0, failed = 0, batches = 0, batched_views = 0;
  double pixels = 0.0, t_first = 0.0, t_last = 0.0;
};

namespace {

// Binning memory per pixel of a view: pair buffers (4 x 4 B per pair) for an
// assumed 32 pairs per pixel, plus records and sort temporaries per splat.
size_t request_cost(const ts_scene* s, const ts_camera& c, int64_t n) {
  const size_t px = (size_t)c.width * c.height;
  return px * 16 + px * 32 * 16 + (size_t)n * 160;
}

void worker_loop(ts_server* sv, int w) {
  cudaSetDevice(sv->device);
  cudaStream_t st = sv->streams[w];
  cudaEvent_t ev;
  cudaEventCreateWithFlags(&ev, cudaEventBlockingSync | cudaEventDisableTiming);
  std::vector<Request*> batch;
  std::vector<ts_scene*> scenes;
  std::vector<ts_camera> cams;
  std::vector<float*> outs;
  for (;;) {
    batch.clear();
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv_work.wait(lk, [&] {
        return sv->stop || (!sv->queue.empty() && sv->inflight + sv->queue.front()->cost <= sv->arena);
      });
      if (sv->stop && sv->queue.empty()) break;
      if (sv->stop) break;
      const int dtype = sv->queue.front()->dtype;
      while (!sv->queue.empty() && (int)batch.size() < sv->max_batch) {
        Request* r = sv->queue.front();
        if (r->dtype != dtype || sv->inflight + r->cost > sv->arena) break;
        sv->queue.pop_front();
        sv->inflight += r->cost;
        r->state = 1;
        batch.push_back(r);
      }
    }
    if (batch.empty()) continue;
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
    if (st_all == TS_OK) {
      st_all = ts_render_views(scenes.data(), cams.data(), (int)batch.size(), outs.data(), nullptr, st);
      if (st_all != TS_OK) err = ts_last_error();
    }
    if (st_all == TS_OK && (cudaEventRecord(ev, st) != cudaSuccess || cudaEventSynchronize(ev) != cudaSuccess)) {
      st_all = TS_ERR_CUDA;
      err = "server: batch completion wait failed";
    }
    const double t = now_s();
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      ++sv->batches;
      sv->batched_views += (int64_t)batch.size();
      for (Request* r : batch) {
        r->t_done = t;
        r->status = st_all;
        r->err = err;
        r->state = st_all == TS_OK ? 2 : 3;
        sv->inflight -= (r->cost - r->out_bytes);  // the output stays until collected
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
  r->cost = request_cost(scene, *cam, n);
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
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
  {
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
  return TS_OK;
}

ts_status ts_server_reset_stats(ts_server* sv) {
  if (!sv) return ts::set_error(TS_ERR_ARG, "ts_server_reset_stats: NULL server");
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->lat_ms.clear();
  sv->submitted = sv->completed = sv->rejected = sv->failed = sv->batches = sv->batched_views = 0;
  sv->pixels = 0.0;
  // the throughput window starts now (or at the next submission)
  sv->t_first = now_s();
  sv->t_last = 0.0;
  return TS_OK;
}

}  // extern "C"
