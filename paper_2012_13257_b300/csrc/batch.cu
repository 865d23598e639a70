// Batched forward: B independent images of uneven size through one binning
// pass and one persistent gather over the work items of all their tiles.
//
// The per-image geometry lives in a device descriptor table and the batch
// totals in a small device header, both uploaded from pinned staging with one
// copy; kernel grids are sized from the plan's capacities and the kernels
// read the real totals from the device.  The launch sequence is therefore the
// same for every batch within capacity and is captured once into a CUDA graph
// (per staging slot) and replayed.  Two staging slots alternate so that the
// host can fill the next batch's table while the previous batch runs.
#include <string.h>

#include <mutex>
#include <vector>

#include "api_internal.h"
#include "bwd_args.h"

namespace gmi {

struct BatchSlot {
  char* host = nullptr;             // pinned: totals header + descriptor table
  char* dev = nullptr;              // device copy (inside the plan's allocation)
  cudaEvent_t done = nullptr;       // recorded after the slot's last launch
  cudaGraphExec_t exec = nullptr;   // captured launch sequence (use_graph)
  bool used = false;
};

}  // namespace gmi

struct gmi_batch_plan {
  int device = 0;
  int max_images = 0;
  long long max_points = 0, max_pixels = 0;
  int C = 3;
  gmi_params params;
  int mth = 4, mtw = 4;
  long long cap_nb = 0, cap_mt = 0, cap_wt = 0, cap_ch = 0, cap_sat = 0;
  gmi::WsLayout L;
  void* base = nullptr;             // one device allocation: workspace + tables
  size_t base_bytes = 0;
  size_t stage_bytes = 0;
  gmi::BatchSlot slot[2];
  int next = 0;
  cudaStream_t cap_stream = nullptr; // private stream the launch sequence is captured on
  // backward pass: per-pixel planes, fallback queue and its own staging
  char* bwd_base = nullptr;
  size_t bwd_bytes = 0;
  float4* pplane = nullptr;
  unsigned* fbflag = nullptr;
  uint2* fbq = nullptr;
  // two pinned host buffers for the backward's tables, so that one call's
  // table can be written while the previous call's upload is pending; one
  // device copy (calls on a plan are ordered on one stream)
  char* bwd_host[2] = {nullptr, nullptr};
  char* bwd_dev = nullptr;
  size_t bwd_stage = 0;
  cudaEvent_t bwd_done[2] = {nullptr, nullptr};
  bool bwd_used[2] = {false, false};
  int bwd_next = 0;
  std::mutex mu;
};

namespace gmi {

static size_t stage_size(int max_images) {
  return (size_t)kTotCount * sizeof(long long) + sizeof(ImageGeom) * (size_t)max_images;
}

static size_t bwd_stage_size(int max_images) {
  return stage_size(max_images) + sizeof(BwdImage) * (size_t)max_images;
}

static size_t al256(size_t v) { return (v + 255) / 256 * 256; }

// Geometry of image i of a batch (bases from the running totals).
static void batch_geom(ImageGeom& g, const gmi_batch_plan* p, long long N, int H, int W, float sigma, int bin_px,
                       long long* npt, long long* nb, long long* nwt, long long* nch, long long* nmt, long long* npx,
                       long long* nsat, long long* nsj) {
  memset(&g, 0, sizeof(g));
  fill_geom(g, N, H, W, sigma, p->params.radius_sigmas, bin_px > 0 ? bin_px : p->params.bin_px, p->mth, p->mtw);
  g.pt_base = *npt;
  g.bin_base = *nb;
  g.wt_base = *nwt;
  g.ch_base = *nch;
  g.mt_base = *nmt;
  g.px_base = *npx;
  g.sat_base = *nsat;
  g.satj_base = *nsj;
  *nsat += sat_entries(g);
  *nsj += sat_jobs(g);
  *npt += N;
  *nb += (long long)g.nbx * g.nby;
  *nwt += (long long)g.wtx * g.wty;
  *nch += (N + kChunk - 1) / kChunk;
  *nmt += (long long)g.mtx * g.mty;
  *npx += (long long)H * W;
}

}  // namespace gmi

using namespace gmi;

namespace gmi {
void batch_plan_workspace(const gmi_batch_plan* p, void** base, const WsLayout** L) {
  *base = p->base;
  *L = &p->L;
}
}  // namespace gmi

extern "C" gmi_status gmi_batch_plan_create(int max_images, int64_t max_points, int64_t max_pixels, int C,
                                            const gmi_params* params, gmi_batch_plan** out) {
  if (!out) return GMI_ERR_INVALID_ARG;
  *out = nullptr;
  gmi_status st = check_params(params);
  if (st != GMI_OK) return st;
  if (max_images < 1 || max_points < 0 || max_pixels < 1 || max_points > (1LL << 31) || max_pixels > (1LL << 34))
    return GMI_ERR_INVALID_ARG;
  if (C < 1 || C > kMaxC) return GMI_ERR_UNSUPPORTED;
  gmi_batch_plan* p = new gmi_batch_plan();
  p->max_images = max_images;
  p->max_points = max_points;
  p->max_pixels = max_pixels;
  p->C = C;
  p->params = *params;
  variant_dims(params->variant, &p->mth, &p->mtw);
  // capacities (checked exactly against every batch)
  p->cap_nb = max_pixels + max_images;
  p->cap_mt = max_pixels / (p->mth * p->mtw) * 2 + 64LL * max_images + 1024;
  p->cap_wt = p->cap_mt / 32 * 2 + 8LL * max_images + 64;
  p->cap_ch = (max_points + kChunk - 1) / kChunk + max_images;
  // sum over images of (nby + 1)(nbx + 1) <= bins + pixels + 2 images (nby + nbx <= H W + 1)
  p->cap_sat = p->cap_nb + max_pixels + 2LL * max_images;
  p->L = ws_layout(max_points, p->cap_nb, p->cap_mt, p->cap_wt, p->cap_sat, slot_bytes_for(p->mth, p->mtw, C), 0);
  p->stage_bytes = (stage_size(max_images) + 255) / 256 * 256;
  p->base_bytes = p->L.total + 2 * p->stage_bytes;
  if (cudaGetDevice(&p->device) != cudaSuccess || cudaMalloc(&p->base, p->base_bytes) != cudaSuccess ||
      cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    if (p->base) cudaFree(p->base);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    delete p;
    return GMI_ERR_CUDA;
  }
  // backward regions (planes over all pixels, fallback queue, staging)
  const size_t planes = al256(sizeof(float4) * (size_t)max_pixels * (C == 4 ? 2 : 1));
  p->bwd_stage = al256(bwd_stage_size(max_images));
  p->bwd_bytes = planes + al256(sizeof(unsigned) * (size_t)p->cap_mt) + al256(sizeof(uint2) * (size_t)p->cap_mt) +
                 p->bwd_stage;
  if (cudaMalloc((void**)&p->bwd_base, p->bwd_bytes) != cudaSuccess ||
      cudaMallocHost((void**)&p->bwd_host[0], p->bwd_stage) != cudaSuccess ||
      cudaMallocHost((void**)&p->bwd_host[1], p->bwd_stage) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->bwd_done[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->bwd_done[1], cudaEventDisableTiming) != cudaSuccess) {
    gmi_batch_plan_destroy(p);
    return GMI_ERR_CUDA;
  }
  p->pplane = (float4*)p->bwd_base;
  p->fbflag = (unsigned*)(p->bwd_base + planes);
  p->fbq = (uint2*)(p->bwd_base + planes + al256(sizeof(unsigned) * (size_t)p->cap_mt));
  p->bwd_dev = p->bwd_base + planes + al256(sizeof(unsigned) * (size_t)p->cap_mt) + al256(sizeof(uint2) * (size_t)p->cap_mt);
  for (int k = 0; k < 2; ++k) {
    p->slot[k].dev = (char*)p->base + p->L.total + k * p->stage_bytes;
    if (cudaMallocHost((void**)&p->slot[k].host, p->stage_bytes) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->slot[k].done, cudaEventDisableTiming) != cudaSuccess) {
      gmi_batch_plan_destroy(p);
      return GMI_ERR_CUDA;
    }
    memset(p->slot[k].host, 0, p->stage_bytes);
  }
  *out = p;
  return GMI_OK;
}

extern "C" gmi_status gmi_batch_plan_destroy(gmi_batch_plan* p) {
  if (!p) return GMI_OK;
  for (int k = 0; k < 2; ++k) {
    if (p->slot[k].done) {
      cudaEventSynchronize(p->slot[k].done);
      cudaEventDestroy(p->slot[k].done);
    }
    if (p->slot[k].exec) cudaGraphExecDestroy(p->slot[k].exec);
    if (p->slot[k].host) cudaFreeHost(p->slot[k].host);
  }
  if (p->base) cudaFree(p->base);
  for (int k = 0; k < 2; ++k) {
    if (p->bwd_done[k]) {
      cudaEventSynchronize(p->bwd_done[k]);
      cudaEventDestroy(p->bwd_done[k]);
    }
  }
  if (p->bwd_base) cudaFree(p->bwd_base);
  for (int k = 0; k < 2; ++k)
    if (p->bwd_host[k]) cudaFreeHost(p->bwd_host[k]);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  delete p;
  return GMI_OK;
}

extern "C" size_t gmi_batch_plan_bytes(const gmi_batch_plan* p) { return p ? p->base_bytes + p->bwd_bytes : 0; }

extern "C" gmi_status gmi_forward_batched(gmi_batch_plan* p, const gmi_image_desc* descs, int B, int use_graph,
                                          gmi_stream_t stream) {
  if (!p || (B > 0 && !descs) || B < 0) return GMI_ERR_INVALID_ARG;
  if (B > p->max_images) return GMI_ERR_CAPACITY;
  cudaStream_t s = (cudaStream_t)stream;
  for (int i = 0; i < B; ++i) {
    const gmi_image_desc& d = descs[i];
    if (d.N < 0 || d.H < 1 || d.W < 1 || (long long)d.H * d.W > (1LL << 31) || !d.image) return GMI_ERR_INVALID_ARG;
    if (!(isfinite(d.sigma) && d.sigma > 0.0f) || d.bin_px < 0 || d.bin_px > 1024) return GMI_ERR_INVALID_ARG;
    if (d.N > 0 && (!d.points || !d.values)) return GMI_ERR_INVALID_ARG;
    if (((uintptr_t)d.points & 7u) || ((uintptr_t)d.values & 3u) || ((uintptr_t)d.image & 3u)) return GMI_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(p->mu);
  const int k = p->next;
  p->next ^= 1;
  BatchSlot& sl = p->slot[k];
  if (sl.used && cudaEventSynchronize(sl.done) != cudaSuccess) return GMI_ERR_CUDA;   // staging free again

  long long* tot = (long long*)sl.host;
  ImageGeom* table = (ImageGeom*)(sl.host + kTotCount * sizeof(long long));
  long long npt = 0, nb = 0, nwt = 0, nch = 0, nmt = 0, npx = 0, nsat = 0, nsj = 0;
  for (int i = 0; i < B; ++i) {
    const gmi_image_desc& d = descs[i];
    ImageGeom& g = table[i];
    batch_geom(g, p, d.N, d.H, d.W, d.sigma, d.bin_px, &npt, &nb, &nwt, &nch, &nmt, &npx, &nsat, &nsj);
    g.points = d.points;
    g.values = d.values;
    g.image = d.image;
    g.den = d.den;
    g.shift = d.shift;
    set_vec_ok(g);
  }
  if (npt > p->max_points || nb > p->cap_nb || nwt > p->cap_wt || nch > p->cap_ch || nmt > p->cap_mt ||
      npx > p->max_pixels || nsat > p->cap_sat)
    return GMI_ERR_CAPACITY;
  tot[kTotImages] = B;
  tot[kTotPoints] = npt;
  tot[kTotBins] = nb;
  tot[kTotWarpTiles] = nwt;
  tot[kTotChunks] = nch;
  tot[kTotMicroTiles] = nmt;
  tot[kTotPixels] = npx;
  tot[kTotSatJobs] = nsj;

  KArgs a;
  memset(&a, 0, sizeof(a));
  a.gather = p->params.gather;
  a.w = bind_ws(p->base, p->L);
  a.w.table = (const ImageGeom*)(sl.dev + kTotCount * sizeof(long long));
  a.totals = (const long long*)sl.dev;
  a.n_images = p->max_images;
  a.C = p->C;
  a.n_total = p->max_points;   // grid sizes: capacities
  a.nb_total = p->cap_nb;
  a.wt_total = p->cap_wt;
  a.ch_total = p->cap_ch;
  a.mt_total = p->cap_mt;
  a.satj_total = nsj;   // read from the device totals at run time
  const bool trunc = p->params.mode == GMI_MODE_TRUNCATED;
  const size_t copy_bytes = stage_size(p->max_images);

  if (use_graph) {
    if (!sl.exec) {
      // captured on the plan's own stream (the caller's may be the legacy
      // default stream, which cannot be captured); replayed on the caller's
      cudaGraph_t graph = nullptr;
      cudaStream_t cs = p->cap_stream;
      warm_near_caches(p->mth, p->mtw, p->C, trunc, 0, p->params.gather);   // host caches, outside the capture
      if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return GMI_ERR_CUDA;
      cudaError_t e = cudaMemcpyAsync(sl.dev, sl.host, copy_bytes, cudaMemcpyHostToDevice, cs);
      gmi_status st = e == cudaSuccess ? run_forward_pipeline(a, p->L, p->base, p->mth, p->mtw, trunc, cs) : GMI_ERR_CUDA;
      const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
      if (st != GMI_OK || ec != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return st != GMI_OK ? st : GMI_ERR_CUDA;
      }
      const cudaError_t ei = cudaGraphInstantiate(&sl.exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ei != cudaSuccess) {
        sl.exec = nullptr;
        return GMI_ERR_CUDA;
      }
    }
    if (cudaGraphLaunch(sl.exec, s) != cudaSuccess) return GMI_ERR_CUDA;
  } else {
    if (cudaMemcpyAsync(sl.dev, sl.host, copy_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return GMI_ERR_CUDA;
    gmi_status st = run_forward_pipeline(a, p->L, p->base, p->mth, p->mtw, trunc, s);
    if (st != GMI_OK) return st;
  }
  if (cudaEventRecord(sl.done, s) != cudaSuccess) return GMI_ERR_CUDA;
  sl.used = true;
  return (p->params.flags & GMI_FLAG_SYNC_CHECK) ? read_status(p->base, s) : GMI_OK;
}

extern "C" gmi_status gmi_backward_batched(gmi_batch_plan* p, const gmi_grad_desc* descs, int B, gmi_stream_t stream) {
  if (!p || (B > 0 && !descs) || B < 0) return GMI_ERR_INVALID_ARG;
  if (B > p->max_images) return GMI_ERR_CAPACITY;
  cudaStream_t s = (cudaStream_t)stream;
  for (int i = 0; i < B; ++i) {
    const gmi_grad_desc& d = descs[i];
    if (d.N < 0 || d.H < 1 || d.W < 1 || (long long)d.H * d.W > (1LL << 31)) return GMI_ERR_INVALID_ARG;
    if (!d.image || !d.den || !d.shift || !d.grad_image) return GMI_ERR_INVALID_ARG;
    if (!(isfinite(d.sigma) && d.sigma > 0.0f) || d.bin_px < 0 || d.bin_px > 1024) return GMI_ERR_INVALID_ARG;
    if (d.N > 0 && (!d.points || !d.values)) return GMI_ERR_INVALID_ARG;
    if (((uintptr_t)d.points & 7u) || ((uintptr_t)d.values & 3u)) return GMI_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(p->mu);
  const int hs = p->bwd_next;
  char* host = p->bwd_host[hs];
  if (p->bwd_used[hs] && cudaEventSynchronize(p->bwd_done[hs]) != cudaSuccess) return GMI_ERR_CUDA;   // buffer free
  long long* tot = (long long*)host;
  ImageGeom* table = (ImageGeom*)(host + kTotCount * sizeof(long long));
  BwdImage* btab = (BwdImage*)(host + stage_size(p->max_images));
  long long npt = 0, nb = 0, nwt = 0, nch = 0, nmt = 0, npx = 0, nsat = 0, nsj = 0;
  for (int i = 0; i < B; ++i) {
    const gmi_grad_desc& d = descs[i];
    ImageGeom& g = table[i];
    batch_geom(g, p, d.N, d.H, d.W, d.sigma, d.bin_px, &npt, &nb, &nwt, &nch, &nmt, &npx, &nsat, &nsj);
    g.points = d.points;
    g.values = d.values;
    BwdImage& bi = btab[i];
    bi.image = d.image;
    bi.den = d.den;
    bi.shift = d.shift;
    bi.grad = d.grad_image;
    bi.gpts = d.grad_points;
    bi.gvals = d.grad_values;
    bi.gsig = d.grad_sigma;
    bi.inv_s2 = (float)(1.0 / ((double)d.sigma * d.sigma));
    bi.inv_s3 = (float)(1.0 / ((double)d.sigma * d.sigma * d.sigma));
  }
  if (npt > p->max_points || nb > p->cap_nb || nwt > p->cap_wt || nch > p->cap_ch || nmt > p->cap_mt ||
      npx > p->max_pixels || nsat > p->cap_sat)
    return GMI_ERR_CAPACITY;
  tot[kTotImages] = B;
  tot[kTotPoints] = npt;
  tot[kTotBins] = nb;
  tot[kTotWarpTiles] = nwt;
  tot[kTotChunks] = nch;
  tot[kTotMicroTiles] = nmt;
  tot[kTotPixels] = npx;
  tot[kTotSatJobs] = nsj;
  if (cudaMemcpyAsync(p->bwd_dev, host, bwd_stage_size(p->max_images), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return GMI_ERR_CUDA;

  KArgs a;
  memset(&a, 0, sizeof(a));
  a.gather = p->params.gather;
  a.w = bind_ws(p->base, p->L);
  a.w.table = (const ImageGeom*)(p->bwd_dev + kTotCount * sizeof(long long));
  a.w.pplane = p->pplane;
  a.w.fbflag = p->fbflag;
  a.w.fbq = p->fbq;
  a.totals = (const long long*)p->bwd_dev;
  a.n_images = p->max_images;
  a.C = p->C;
  a.n_total = p->max_points;   // grid sizes: capacities
  a.nb_total = p->cap_nb;
  a.wt_total = p->cap_wt;
  a.ch_total = p->cap_ch;
  a.mt_total = p->cap_mt;
  a.px_total = p->max_pixels;
  const bool trunc = p->params.mode == GMI_MODE_TRUNCATED;
  gmi_status st = run_bin_and_plan(a, p->L, p->base, p->mth, p->mtw, trunc, s, false);
  if (st != GMI_OK) return st;
  BwdArgs b;
  memset(&b, 0, sizeof(b));
  b.table = (const BwdImage*)(p->bwd_dev + stage_size(p->max_images));
  b.trunc = trunc ? 1 : 0;
  const ProfileMark pm = profile_begin(GMI_STAGE_BACKWARD, s);
  if (launch_backward(a, b, s) != cudaSuccess) return GMI_ERR_CUDA;
  profile_end(pm, s);
  if (cudaEventRecord(p->bwd_done[hs], s) != cudaSuccess) return GMI_ERR_CUDA;
  p->bwd_used[hs] = true;
  p->bwd_next = hs ^ 1;
  return (p->params.flags & GMI_FLAG_SYNC_CHECK) ? read_status(p->base, s) : GMI_OK;
}

// Equal-shaped (stacked) batches: the descriptor tables built here from base
// pointers and strides, so that a caller holding [B, ...] tensors passes
// their addresses instead of building B descriptors itself.
extern "C" gmi_status gmi_forward_stacked(gmi_batch_plan* p, const float* points, const float* values, int B,
                                          int64_t N, int H, int W, const float* sigmas, float* image, float* den,
                                          float* shift, int use_graph, gmi_stream_t stream) {
  if (!p || !sigmas || B < 1 || B > p->max_images || N < 0 || H < 1 || W < 1 || !image)
    return GMI_ERR_INVALID_ARG;
  const long long px = (long long)H * W;
  std::vector<gmi_image_desc> d((size_t)B);
  for (int i = 0; i < B; ++i) {
    gmi_image_desc& e = d[(size_t)i];
    memset(&e, 0, sizeof(e));
    e.points = points ? points + (size_t)i * N * 2 : nullptr;
    e.values = values ? values + (size_t)i * N * p->C : nullptr;
    e.image = image + (size_t)i * px * p->C;
    e.den = den ? den + (size_t)i * px : nullptr;
    e.shift = shift ? shift + (size_t)i * px : nullptr;
    e.N = N;
    e.H = H;
    e.W = W;
    e.sigma = sigmas[i];
  }
  return gmi_forward_batched(p, d.data(), B, use_graph, stream);
}

extern "C" gmi_status gmi_backward_stacked(gmi_batch_plan* p, const float* points, const float* values, int B,
                                           int64_t N, int H, int W, const float* sigmas, const float* image,
                                           const float* den, const float* shift, const float* grad_image,
                                           float* grad_points, float* grad_values, float* grad_sigma,
                                           gmi_stream_t stream) {
  if (!p || !sigmas || B < 1 || B > p->max_images || N < 0 || H < 1 || W < 1 || !image || !den || !shift ||
      !grad_image)
    return GMI_ERR_INVALID_ARG;
  const long long px = (long long)H * W;
  std::vector<gmi_grad_desc> d((size_t)B);
  for (int i = 0; i < B; ++i) {
    gmi_grad_desc& e = d[(size_t)i];
    memset(&e, 0, sizeof(e));
    e.points = points ? points + (size_t)i * N * 2 : nullptr;
    e.values = values ? values + (size_t)i * N * p->C : nullptr;
    e.image = image + (size_t)i * px * p->C;
    e.den = den + (size_t)i * px;
    e.shift = shift + (size_t)i * px;
    e.grad_image = grad_image + (size_t)i * px * p->C;
    e.grad_points = grad_points ? grad_points + (size_t)i * N * 2 : nullptr;
    e.grad_values = grad_values ? grad_values + (size_t)i * N * p->C : nullptr;
    e.grad_sigma = grad_sigma ? grad_sigma + i : nullptr;
    e.N = N;
    e.H = H;
    e.W = W;
    e.sigma = sigmas[i];
  }
  return gmi_backward_batched(p, d.data(), B, stream);
}
