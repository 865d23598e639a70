// Serving loop with continuous batching (host C++ around the batched forward).
//
//   submit()  -> pending FIFO (host buffers, arrival time stamped)
//   launcher  -> admits pending requests in order while their device footprint
//                fits the memory budget (first-fit pool) and the batch limits,
//                uploads them, runs one batched forward (CUDA-graph replay) on
//                a free stream slot, downloads the images, records an event;
//                up to n_streams batches are on the GPU at once, so requests
//                arriving meanwhile form the next batch and overlap with it
//   completer -> waits for batch events in launch order, stamps completion,
//                frees device memory, wakes waiters
// One device allocation of budget_bytes holds the batch plans' workspaces and
// every admitted request's points, values and image.
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
  Clock::time_point t_submit, t_done;
  size_t off = 0, bytes = 0;     // device region (points | values | image)
  bool done = false;
  gmi_status status = GMI_OK;
};

struct Inflight {
  int slot;
  cudaEvent_t ev;
  std::vector<Request*> reqs;
};

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
  std::thread launcher, completer;

  size_t footprint(const Request& r) const {
    return align256((size_t)r.N * 8) + align256((size_t)r.N * cfg.C * 4) + align256((size_t)r.H * r.W * cfg.C * 4);
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
          if (!pool->alloc(r->bytes, &r->off)) break;   // wait for memory to free up
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
      float* dp = (float*)b;
      float* dv = (float*)(b + align256((size_t)r->N * 8));
      float* di = (float*)(b + align256((size_t)r->N * 8) + align256((size_t)r->N * cfg.C * 4));
      if (r->N > 0) {
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
      if (cudaMemcpyAsync(r->image, descs[i].image, (size_t)r->H * r->W * cfg.C * 4, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess)
        st = GMI_ERR_CUDA;
    }
    cudaEventRecord(events[slot], s);

    lk.lock();
    for (Request* r : batch) r->status = st;
    inflight.push_back(Inflight{slot, events[slot], batch});
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
    Inflight f = inflight.front();
    inflight.pop_front();
    lk.unlock();
    const cudaError_t e = cudaEventSynchronize(f.ev);
    const auto now = Clock::now();
    lk.lock();
    for (Request* r : f.reqs) {
      if (e != cudaSuccess) r->status = GMI_ERR_CUDA;
      r->t_done = now;
      r->done = true;
      pool->release(r->off, r->bytes);
      n_completed += 1;
      n_pixels += (uint64_t)r->H * r->W;
    }
    slot_busy[f.slot] = false;
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

gmi_status gmi_server_submit(gmi_server* s, const float* points, const float* values, int64_t N, int H, int W,
                             float sigma, float* image, uint64_t* id) {
  if (!s || !id || !image || N < 0 || H < 1 || W < 1 || !(sigma > 0.0f) || !(sigma < 3.0e38f) ||
      (N > 0 && (!points || !values)))
    return GMI_ERR_INVALID_ARG;
  if ((int64_t)H * W > s->cfg.max_batch_pixels || N > s->max_batch_points) return GMI_ERR_CAPACITY;
  Request* r = new Request();
  r->points = points;
  r->values = values;
  r->image = image;
  r->N = N;
  r->H = H;
  r->W = W;
  r->sigma = sigma;
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
  delete s->pool;
  delete s;
  return GMI_OK;
}

}  // extern "C"
