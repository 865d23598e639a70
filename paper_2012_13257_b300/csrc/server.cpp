// Serving loop with continuous batching (host C++ around the batched forward).
//
//   submit()  -> pending FIFO (host buffers, arrival time stamped)
//   launcher  -> admits pending requests in order while their device footprint
//                fits the memory budget (first-fit pool) and the batch limits,
//                uploads them, runs one batched forward (CUDA-graph replay) on
//                a free stream slot, downloads the images, records an event;
//                up to n_streams batches are on the GPU at once, so requests
//                arriving meanwhile form the next batch and overlap with it
//   completer -> polls the events of every batch in flight (a short batch on
//                one stream slot completes before a long one launched earlier
//                on another), stamps each batch's completion when its event
//                is seen, frees device memory, wakes waiters, and appends one
//                JSON line per request to the log when one is set
// One device allocation of budget_bytes holds the batch plans' workspaces and
// every admitted request's points, values and image.  Requests submitted with
// device buffers are read and written in place and take none of the pool.
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "gmi.h"

namespace {

using Clock = std::chrono::steady_clock;

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// First-fit allocator over [0, size) of the device pool.
class Pool {
 public:
  explicit Pool(size_t size) { free_[0] = size; }
  bool alloc(size_t n, size_t* off) {
    n = align256(n);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n, start = it->first + n;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += n;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = align256(n);
    used_ -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0;
};

struct Request {
  uint64_t id;
  const float* points;
  const float* values;
  float* image;
  int64_t N;
  int H, W;
  float sigma;
  bool on_device = false;        // buffers are device memory (no copies, no pool region)
  Clock::time_point t_submit, t_admit, t_launch, t_done;
  uint64_t batch = 0;
  int slot = -1;
  size_t off = 0, bytes = 0;     // device region (points | values | image)
  bool done = false;
  gmi_status status = GMI_OK;
};

struct Inflight {
  int slot;
  cudaEvent_t ev;
  std::vector<Request*> reqs;
};

double secs(Clock::time_point a, Clock::time_point b) { return std::chrono::duration<double>(b - a).count(); }

}  // namespace

struct gmi_server {
  gmi_server_config cfg;
  int device = 0;
  char* dev_base = nullptr;
  size_t req_bytes = 0;               // part of the budget for request data
  Pool* pool = nullptr;
  std::vector<gmi_batch_plan*> plans;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  std::vector<bool> slot_busy;
  int64_t max_batch_points = 0;

  std::mutex mu;
  std::condition_variable cv_launch, cv_done, cv_complete;
  std::deque<Request*> pending;
  std::deque<Inflight> inflight;
  std::unordered_map<uint64_t, Request*> reqs;
  uint64_t next_id = 1;
  bool stop = false;
  bool launching = false;             // the launcher holds a batch it has not queued yet
  uint64_t n_completed = 0, n_launches = 0, n_pixels = 0;
  int max_in_flight = 0;
  Clock::time_point t0 = Clock::now();   // origin of the log's times
  FILE* log = nullptr;
  std::thread launcher, completer;

  size_t footprint(const Request& r) const {
    if (r.on_device) return 0;
    return align256((size_t)r.N * 8) + align256((size_t)r.N * cfg.C * 4) + align256((size_t)r.H * r.W * cfg.C * 4);
  }
  void log_request(const Request& r) {
    if (!log) return;
    fprintf(log,
            "{\"id\": %llu, \"device\": %d, \"N\": %lld, \"H\": %d, \"W\": %d, \"batch\": %llu, \"slot\": %d, "
            "\"submit\": %.7f, \"admit\": %.7f, \"launch\": %.7f, \"done\": %.7f, \"status\": %d}\n",
            (unsigned long long)r.id, r.on_device ? 1 : 0, (long long)r.N, r.H, r.W, (unsigned long long)r.batch,
            r.slot, secs(t0, r.t_submit), secs(t0, r.t_admit), secs(t0, r.t_launch), secs(t0, r.t_done),
            (int)r.status);
  }

  void launcher_loop();
  void completer_loop();
};

void gmi_server::launcher_loop() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    // a free stream slot and at least one admissible request
    int slot = -1;
    std::vector<Request*> batch;
    for (;;) {
      if (stop && pending.empty()) return;
      slot = -1;
      for (size_t k = 0; k < slot_busy.size(); ++k)
        if (!slot_busy[k]) {
          slot = (int)k;
          break;
        }
      if (slot >= 0 && !pending.empty()) {
        int64_t px = 0, pts = 0;
        while (!pending.empty() && (int)batch.size() < cfg.max_batch_images) {
          Request* r = pending.front();
          const int64_t rpx = (int64_t)r->H * r->W;
          if (!batch.empty() && (px + rpx > cfg.max_batch_pixels || pts + r->N > max_batch_points)) break;
          if (r->bytes > 0 && !pool->alloc(r->bytes, &r->off)) break;   // wait for memory to free up
          r->t_admit = Clock::now();
          pending.pop_front();
          batch.push_back(r);
          px += rpx;
          pts += r->N;
        }
        if (!batch.empty()) break;
      }
      cv_launch.wait(lk);
    }
    slot_busy[slot] = true;
    launching = true;
    lk.unlock();

    cudaStream_t s = streams[slot];
    std::vector<gmi_image_desc> descs(batch.size());
    gmi_status st = GMI_OK;
    for (size_t i = 0; i < batch.size(); ++i) {
      Request* r = batch[i];
      char* b = dev_base + r->off;
      float* dp = r->on_device ? (float*)r->points : (float*)b;
      float* dv = r->on_device ? (float*)r->values : (float*)(b + align256((size_t)r->N * 8));
      float* di = r->on_device ? r->image
                               : (float*)(b + align256((size_t)r->N * 8) + align256((size_t)r->N * cfg.C * 4));
      if (r->N > 0 && !r->on_device) {
        if (cudaMemcpyAsync(dp, r->points, (size_t)r->N * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(dv, r->values, (size_t)r->N * cfg.C * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
          st = GMI_ERR_CUDA;
      }
      gmi_image_desc& d = descs[i];
      memset(&d, 0, sizeof(d));
      d.points = dp;
      d.values = dv;
      d.image = di;
      d.N = r->N;
      d.H = r->H;
      d.W = r->W;
      d.sigma = r->sigma;
    }
    if (st == GMI_OK) st = gmi_forward_batched(plans[slot], descs.data(), (int)descs.size(), 1, (gmi_stream_t)s);
    for (size_t i = 0; i < batch.size() && st == GMI_OK; ++i) {
      Request* r = batch[i];
      if (r->on_device) continue;
      if (cudaMemcpyAsync(r->image, descs[i].image, (size_t)r->H * r->W * cfg.C * 4, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess)
        st = GMI_ERR_CUDA;
    }
    cudaEventRecord(events[slot], s);

    const auto t_launch = Clock::now();
    lk.lock();
    for (Request* r : batch) {
      r->status = st;
      r->t_launch = t_launch;
      r->batch = n_launches;
      r->slot = slot;
    }
    inflight.push_back(Inflight{slot, events[slot], batch});
    if ((int)inflight.size() > max_in_flight) max_in_flight = (int)inflight.size();
    launching = false;
    n_launches += 1;
    cv_complete.notify_all();
  }
}

void gmi_server::completer_loop() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    while (inflight.empty()) {
      if (stop && pending.empty() && !launching) return;
      cv_complete.wait(lk);
    }
    // every batch in flight whose event has completed (any order); when none
    // has, look again shortly (the stamp is within that interval of the
    // event's completion)
    std::vector<Inflight> finished;
    std::vector<cudaError_t> errs;
    for (auto it = inflight.begin(); it != inflight.end();) {
      const cudaError_t q = cudaEventQuery(it->ev);
      if (q == cudaErrorNotReady) {
        ++it;
        continue;
      }
      finished.push_back(*it);
      errs.push_back(q);
      it = inflight.erase(it);
    }
    if (finished.empty()) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
      continue;
    }
    const auto now = Clock::now();
    for (size_t k = 0; k < finished.size(); ++k) {
      for (Request* r : finished[k].reqs) {
        if (errs[k] != cudaSuccess) r->status = GMI_ERR_CUDA;
        r->t_done = now;
        r->done = true;
        if (r->bytes > 0) pool->release(r->off, r->bytes);
        n_completed += 1;
        n_pixels += (uint64_t)r->H * r->W;
        log_request(*r);
      }
      slot_busy[finished[k].slot] = false;
    }
    cv_done.notify_all();
    cv_launch.notify_all();
  }
}

extern "C" {

gmi_status gmi_server_config_default(gmi_server_config* cfg) {
  if (!cfg) return GMI_ERR_INVALID_ARG;
  memset(cfg, 0, sizeof(*cfg));
  cfg->budget_bytes = (size_t)40 << 30;
  cfg->max_batch_images = 64;
  cfg->max_batch_pixels = (int64_t)1 << 25;
  cfg->n_streams = 2;
  cfg->C = 3;
  cfg->radius_sigmas = 6.0f;
  cfg->mode = GMI_MODE_EXACT;
  return GMI_OK;
}

gmi_status gmi_server_create(const gmi_server_config* cfg, gmi_server** out) {
  if (!cfg || !out) return GMI_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->max_batch_images < 1 || cfg->max_batch_pixels < 1 || cfg->n_streams < 1 || cfg->n_streams > 8 ||
      cfg->C < 1 || cfg->C > 4 || !(cfg->radius_sigmas > 0) || (cfg->mode != GMI_MODE_EXACT && cfg->mode != GMI_MODE_TRUNCATED))
    return GMI_ERR_INVALID_ARG;
  gmi_server* s = new gmi_server();
  s->cfg = *cfg;
  s->max_batch_points = 2 * cfg->max_batch_pixels;
  cudaGetDevice(&s->device);
  gmi_params p;
  gmi_params_default(&p);
  p.radius_sigmas = cfg->radius_sigmas;
  p.mode = cfg->mode;
  size_t plan_bytes = 0;
  for (int k = 0; k < cfg->n_streams; ++k) {
    gmi_batch_plan* plan = nullptr;
    gmi_status st = gmi_batch_plan_create(cfg->max_batch_images, s->max_batch_points, cfg->max_batch_pixels, cfg->C,
                                          &p, &plan);
    if (st != GMI_OK) {
      gmi_server_destroy(s);
      return st;
    }
    s->plans.push_back(plan);
    plan_bytes += gmi_batch_plan_bytes(plan);
    cudaStream_t st_;
    cudaEvent_t ev;
    if (cudaStreamCreateWithFlags(&st_, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      gmi_server_destroy(s);
      return GMI_ERR_CUDA;
    }
    s->streams.push_back(st_);
    s->events.push_back(ev);
    s->slot_busy.push_back(false);
  }
  if (plan_bytes >= cfg->budget_bytes) {
    gmi_server_destroy(s);
    return GMI_ERR_BUDGET;
  }
  s->req_bytes = (cfg->budget_bytes - plan_bytes) / 256 * 256;
  if (cudaMalloc((void**)&s->dev_base, s->req_bytes) != cudaSuccess) {
    gmi_server_destroy(s);
    return GMI_ERR_CUDA;
  }
  s->pool = new Pool(s->req_bytes);
  s->launcher = std::thread([s] { s->launcher_loop(); });
  s->completer = std::thread([s] { s->completer_loop(); });
  *out = s;
  return GMI_OK;
}

}  // extern "C"

namespace {

bool on_device_of(const void* p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == device;
}

gmi_status submit_impl(gmi_server* s, const float* points, const float* values, int64_t N, int H, int W,
                       float sigma, float* image, bool on_device, uint64_t* id) {
  if (!s || !id || !image || N < 0 || H < 1 || W < 1 || !(sigma > 0.0f) || !(sigma < 3.0e38f) ||
      (N > 0 && (!points || !values)))
    return GMI_ERR_INVALID_ARG;
  if ((int64_t)H * W > s->cfg.max_batch_pixels || N > s->max_batch_points) return GMI_ERR_CAPACITY;
  if (on_device) {
    if (((uintptr_t)points & 7u) || ((uintptr_t)values & 3u) || ((uintptr_t)image & 3u)) return GMI_ERR_INVALID_ARG;
    if (!on_device_of(image, s->device) || (N > 0 && (!on_device_of(points, s->device) ||
                                                      !on_device_of(values, s->device))))
      return GMI_ERR_INVALID_ARG;
  }
  Request* r = new Request();
  r->points = points;
  r->values = values;
  r->image = image;
  r->N = N;
  r->H = H;
  r->W = W;
  r->sigma = sigma;
  r->on_device = on_device;
  r->bytes = s->footprint(*r);
  if (r->bytes > s->req_bytes) {
    delete r;
    return GMI_ERR_BUDGET;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    delete r;
    return GMI_ERR_INVALID_ARG;
  }
  r->id = s->next_id++;
  r->t_submit = Clock::now();
  s->reqs[r->id] = r;
  s->pending.push_back(r);
  *id = r->id;
  s->cv_launch.notify_all();
  return GMI_OK;
}

}  // namespace

extern "C" {

gmi_status gmi_server_submit(gmi_server* s, const float* points, const float* values, int64_t N, int H, int W,
                             float sigma, float* image, uint64_t* id) {
  return submit_impl(s, points, values, N, H, W, sigma, image, false, id);
}

gmi_status gmi_server_submit_device(gmi_server* s, const float* points, const float* values, int64_t N, int H,
                                    int W, float sigma, float* image, uint64_t* id) {
  return submit_impl(s, points, values, N, H, W, sigma, image, true, id);
}

gmi_status gmi_server_get_counters(gmi_server* s, gmi_server_counters* out) {
  if (!s || !out) return GMI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  memset(out, 0, sizeof(*out));
  out->completed = s->n_completed;
  out->launches = s->n_launches;
  out->pixels = s->n_pixels;
  out->bytes_in_use = s->pool ? s->pool->used() : 0;
  out->in_flight = (int)s->inflight.size();
  out->max_in_flight = s->max_in_flight;
  return GMI_OK;
}

gmi_status gmi_server_set_log(gmi_server* s, const char* path) {
  if (!s) return GMI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->log) {
    fclose(s->log);
    s->log = nullptr;
  }
  if (path) {
    s->log = fopen(path, "w");
    if (!s->log) return GMI_ERR_INVALID_ARG;
  }
  return GMI_OK;
}

gmi_status gmi_server_wait(gmi_server* s, uint64_t id, int timeout_ms, double* latency_s) {
  if (!s) return GMI_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return GMI_ERR_NOT_FOUND;
  Request* r = it->second;
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, [r] { return r->done; });
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [r] { return r->done; })) {
    return GMI_ERR_TIMEOUT;
  }
  const gmi_status st = r->status;
  if (latency_s) latency_s[0] = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  s->reqs.erase(it);
  delete r;
  return st;
}

gmi_status gmi_server_poll(gmi_server* s, uint64_t id) {
  if (!s) return GMI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return GMI_ERR_NOT_FOUND;
  return it->second->done ? GMI_OK : GMI_ERR_TIMEOUT;
}

gmi_status gmi_server_stats(gmi_server* s, uint64_t* completed, uint64_t* launches, uint64_t* pixels,
                            size_t* bytes_in_use) {
  if (!s) return GMI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (completed) *completed = s->n_completed;
  if (launches) *launches = s->n_launches;
  if (pixels) *pixels = s->n_pixels;
  if (bytes_in_use) *bytes_in_use = s->pool ? s->pool->used() : 0;
  return GMI_OK;
}

gmi_status gmi_server_destroy(gmi_server* s) {
  if (!s) return GMI_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_launch.notify_all();
    s->cv_complete.notify_all();
  }
  if (s->launcher.joinable()) s->launcher.join();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->cv_complete.notify_all();
  }
  if (s->completer.joinable()) s->completer.join();
  for (auto& kv : s->reqs) delete kv.second;
  for (gmi_batch_plan* p : s->plans) gmi_batch_plan_destroy(p);
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  for (cudaEvent_t e : s->events) cudaEventDestroy(e);
  if (s->dev_base) cudaFree(s->dev_base);
  if (s->log) fclose(s->log);
  delete s->pool;
  delete s;
  return GMI_OK;
}

}  // extern "C"
