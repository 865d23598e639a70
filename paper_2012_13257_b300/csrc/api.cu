// Host side of the libgmi C ABI: argument checks, workspace layout, and the
// launch sequence of the single-image forward pass
//   memset(status, bin counts) -> bin_count -> scan_partial -> scan_final
//   -> scatter + plan (one launch) -> near gather -> far gather
// (replayed as one cached CUDA graph with GMI_FLAG_GRAPH).  All kernels run
// on the caller's stream; nothing here allocates device memory.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>

#include "api_internal.h"
#include "gmi.h"

namespace gmi {

cudaError_t launch_near(const KArgs& a, int mth, int mtw, bool trunc, int ppk, int grid, cudaStream_t s);
cudaError_t launch_near_staged(const KArgs& a, int mth, int mtw, bool trunc, int grid, cudaStream_t s);
cudaError_t launch_pp_exact_forward(const KArgs& a, int mth, int mtw, int ppk, cudaStream_t s);
void warm_pp_exact(int C, int ppk);
void warm_scatter_plan();
int staged_blocks_per_sm(int mth, int mtw, int C, bool trunc);
cudaError_t launch_scatter_plan(const KArgs& a, bool trunc, int n_scatter, cudaStream_t s);
int near_blocks_per_sm(int mth, int mtw, int C, bool trunc, int ppk);
cudaError_t launch_far(const KArgs& a, int mth, int mtw, int sms, cudaStream_t s);
__global__ void bin_count_kernel(KArgs a);
__global__ void scan_partial_kernel(const unsigned* cnt, long long nb, unsigned* partials, const long long* totals);
__global__ void scan_final_kernel(unsigned* off, long long nb, const unsigned* partials, const long long* totals);
__global__ void scan_one_kernel(unsigned* off, long long nb, unsigned* partials, unsigned* status, unsigned polls);

// Blocks of the one-launch scan that can be resident on the device at once
// (cached; filled before any capture by warm_near_caches).
static int scan_one_capacity() {
  static const int n = [] {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, scan_one_kernel, 256, 0) != cudaSuccess || b < 1) b = 0;
    return b * device_sm_count();
  }();
  return n;
}
__global__ void bin_scatter_kernel(KArgs a);
__global__ void batch_clear_kernel(KArgs a);

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int device_sm_count() {
  static int cache[64];
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  std::lock_guard<std::mutex> lk(mu);
  if (cache[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    cache[dev] = n;
  }
  return cache[dev];
}

void variant_dims(int variant, int* mth, int* mtw) {
  switch (variant) {
    case GMI_VARIANT_MT4x8: *mth = 4; *mtw = 8; break;
    case GMI_VARIANT_MT2x4: *mth = 2; *mtw = 4; break;
    case GMI_VARIANT_MT4x2: *mth = 4; *mtw = 2; break;
    default: *mth = 4; *mtw = 4; break;
  }
}

int auto_bin_px(long long n, int H, int W) {
  if (n <= 0) return 64;
  const double rho = (double)n / ((double)H * (double)W);
  // about one point per bin: b ~ 1/sqrt(rho), rounded to a power of two
  const double l = -0.5 * log2(rho);
  int e = (int)floor(l + 0.5);
  if (e < 0) e = 0;
  if (e > 6) e = 6;
  return 1 << e;
}

gmi_status check_params(const gmi_params* p) {
  if (!p) return GMI_ERR_INVALID_ARG;
  if (!(isfinite(p->sigma) && p->sigma > 0.0f)) return GMI_ERR_INVALID_ARG;
  if (!(isfinite(p->radius_sigmas) && p->radius_sigmas > 0.0f)) return GMI_ERR_INVALID_ARG;
  if (p->mode != GMI_MODE_EXACT && p->mode != GMI_MODE_TRUNCATED) return GMI_ERR_INVALID_ARG;
  if (p->bin_px < 0 || p->bin_px > 1024) return GMI_ERR_INVALID_ARG;
  if (p->variant < 0 || p->variant > GMI_VARIANT_MT4x2) return GMI_ERR_INVALID_ARG;
  if (p->gather < GMI_GATHER_AUTO || p->gather > GMI_GATHER_DIRECT) return GMI_ERR_INVALID_ARG;
  if (p->flags & ~(GMI_FLAG_SYNC_CHECK | GMI_FLAG_GRAPH)) return GMI_ERR_INVALID_ARG;
  return GMI_OK;
}

gmi_status check_shape(long long N, int C, int H, int W) {
  if (N < 0 || H < 1 || W < 1) return GMI_ERR_INVALID_ARG;
  if ((long long)H * (long long)W > (1LL << 31)) return GMI_ERR_INVALID_ARG;
  if (N > (1LL << 31)) return GMI_ERR_INVALID_ARG;
  if (C < 1 || C > kMaxC) return GMI_ERR_UNSUPPORTED;
  return GMI_OK;
}

// Fills the derived fields of an image geometry.
void fill_geom(ImageGeom& g, long long N, int H, int W, float sigma, float k, int bin_px, int mth, int mtw) {
  g.n = N;
  g.H = H;
  g.W = W;
  g.b = bin_px > 0 ? bin_px : auto_bin_px(N, H, W);
  g.inv_b = 1.0f / (float)g.b;
  g.nbx = (W + g.b - 1) / g.b;
  g.nby = (H + g.b - 1) / g.b;
  g.mtx = (W + mtw - 1) / mtw;
  g.mty = (H + mth - 1) / mth;
  g.wtx = (g.mtx + 7) / 8;
  g.wty = (g.mty + 3) / 4;
  g.sigma = sigma;
  const double kappa = 1.4426950408889634 / (2.0 * (double)sigma * (double)sigma);
  g.kappa = (float)kappa;
  g.sk = (float)sqrt(kappa);
  g.r2k = (float)((double)k * k * (double)sigma * sigma);
  g.u_near_max = (float)(100.0 / kappa);
  g.e_trunc = (float)((double)k * k * 1.4426950408889634 / 2.0);
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

void set_vec_ok(ImageGeom& g) {
  g.vec_ok = (g.W % 4 == 0) && aligned16(g.image) && (!g.den || aligned16(g.den)) && (!g.shift || aligned16(g.shift));
}

size_t slot_bytes_for(int mth, int mtw, int C) { return sizeof(float) * 32u * mth * mtw * (C + 1); }

// Workspace layout for totals (points, bins, micro-tiles, warp tiles); bytes.
long long sat_entries(const ImageGeom& g) { return (long long)(g.nby + 1) * (long long)(g.nbx + 1); }
long long sat_jobs(const ImageGeom& g) { return (g.nbx + 1 + 31) / 32; }

WsLayout ws_layout(long long n_total, long long nb_total, long long mt_total, long long wt_total,
                   long long sat_entries, size_t slot_bytes, long long extra_bytes, bool tile_plans) {
  WsLayout L;
  L.guards.n = 0;
  size_t o = 0;
  // the next region of `bytes` (256-byte aligned), and its guard area
  auto region = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, 256);
    if (kGuardBytes > 0 && L.guards.n < kMaxGuards) {
      L.guards.off[L.guards.n++] = o;
      o += kGuardBytes;
    }
    return at;
  };
  L.cap_items = (unsigned)std::min<long long>(wt_total * kSplitMax, 0x7fffffffLL);
  L.cap_slots = (unsigned)std::min<long long>(wt_total > 0 ? wt_total : 1, 0x7fffffffLL);
  L.status = region(sizeof(unsigned) * kStatusWords);
  L.off = region(sizeof(unsigned) * (size_t)(nb_total + 1) + 16);   // (+ slack, as below)
  L.oob = region((size_t)nb_total);
  L.tile_done = region(sizeof(unsigned) * (size_t)(wt_total > 0 ? wt_total : 1));
  L.zero_end = o;                               // [0, zero_end) is cleared per call
  L.rank = region(sizeof(unsigned) * (size_t)n_total);
  // (16 bytes of slack after each sorted array: the staged gather's bulk
  // copies widen their ranges to even indices, one record past the end at most)
  L.sxy = region(sizeof(float2) * (size_t)n_total + 16);
  L.sval = region(sizeof(float4) * (size_t)n_total + 16);
  L.perm = region(sizeof(unsigned) * (size_t)n_total);
  L.spp = region(sizeof(float4) * (size_t)n_total);
  L.partials = region(sizeof(unsigned) * (size_t)((nb_total + kScanChunk - 1) / kScanChunk + 1));
  L.farq = region(sizeof(uint2) * (size_t)(mt_total > 0 ? mt_total : 1));
  L.items = region(sizeof(uint4) * (size_t)(L.cap_items > 0 ? L.cap_items : 1));
  L.slots = region(slot_bytes * (size_t)L.cap_slots);
  L.ubound = region(sizeof(float) * 32u * (size_t)(wt_total > 0 ? wt_total : 1));
  L.sat = region(sizeof(unsigned) * (size_t)(sat_entries > 0 ? sat_entries : 1));
  L.has_tplan = tile_plans;
  L.tplan = region(tile_plans ? sizeof(TilePlanRec) * (size_t)(wt_total > 0 ? wt_total : 1) : 0);
  L.extra = o;  o = align_up(o + (size_t)extra_bytes, 256);
  L.total = o;
  return L;
}

DevWork bind_ws(void* ws, const WsLayout& L) {
  char* b = (char*)ws;
  DevWork w;
  w.status = (unsigned*)(b + L.status);
  w.off = (unsigned*)(b + L.off);
  w.oob = (unsigned char*)(b + L.oob);
  w.rank = (unsigned*)(b + L.rank);
  w.sxy = (float2*)(b + L.sxy);
  w.sval = (float4*)(b + L.sval);
  w.partials = (unsigned*)(b + L.partials);
  w.farq = (uint2*)(b + L.farq);
  w.items = (uint4*)(b + L.items);
  w.tile_done = (unsigned*)(b + L.tile_done);
  w.slots = (float*)(b + L.slots);
  w.ubound = (float*)(b + L.ubound);
  w.perm = (unsigned*)(b + L.perm);
  w.spp = (float4*)(b + L.spp);
  w.sat = (unsigned*)(b + L.sat);
  w.tplan = L.has_tplan ? (TilePlanRec*)(b + L.tplan) : nullptr;
  w.pplane = nullptr;
  w.fbflag = nullptr;
  w.fbq = nullptr;
  w.sig_part = nullptr;
  w.ppmom = nullptr;
  w.table = nullptr;
  return w;
}

// Binning (memset, count, scan, scatter) and, with plan set, the near-kernel
// plan.  Grid sizes come from a's totals; in a batched call (a.totals set)
// they are the plan's capacities and the kernels read the real totals from
// the device.
gmi_status run_bin_and_plan(KArgs& a, const WsLayout& L, void* ws, int mth, int mtw, bool trunc,
                            cudaStream_t s, bool plan) {
  const ProfileMark pb = profile_begin(GMI_STAGE_BIN, s);
  const int sms = device_sm_count();
  if (a.totals) {
    batch_clear_kernel<<<sms * 4, 256, 0, s>>>(a);
  } else if (kGuardBytes == 0) {
    if (cudaMemsetAsync(ws, 0, L.zero_end, s) != cudaSuccess) return GMI_ERR_CUDA;
  } else {
    // checked builds: the cleared regions one by one, around their guards
    const size_t starts[4] = {L.status, L.off, L.oob, L.tile_done};
    for (int k = 0; k < 4; ++k)
      if (cudaMemsetAsync((char*)ws + starts[k], 0, L.guards.off[k] - starts[k], s) != cudaSuccess)
        return GMI_ERR_CUDA;
  }
  if (kGuardBytes > 0 && launch_canaries(ws, L.guards, false, a.w.status, s) != cudaSuccess) return GMI_ERR_CUDA;
  a.cap_items = L.cap_items;
  a.cap_slots = L.cap_slots;
  a.mth = mth;
  a.mtw = mtw;
  int gb = 0;
  if (a.n_total > 0) {
    gb = (int)std::min<long long>(a.ch_total, (long long)sms * 32);
    bin_count_kernel<<<gb, 256, 0, s>>>(a);
    const int ns = (int)((a.nb_total + kScanChunk - 1) / kScanChunk);
    if (!a.totals && ns <= scan_one_capacity()) {
      // single image, every block resident at once: one cooperative launch
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cfg.gridDim = dim3((unsigned)ns);
      cfg.blockDim = dim3(256);
      cfg.stream = s;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      if (cudaLaunchKernelEx(&cfg, scan_one_kernel, a.w.off, (long long)a.nb_total, a.w.partials, a.w.status,
                             scan_wait_polls()) != cudaSuccess)
        return GMI_ERR_CUDA;
    } else {
      scan_partial_kernel<<<ns, 256, 0, s>>>(a.w.off, a.nb_total, a.w.partials, a.totals);
      scan_final_kernel<<<ns, 256, 0, s>>>(a.w.off, a.nb_total, a.w.partials, a.totals);
    }
    if (cudaGetLastError() != cudaSuccess) return GMI_ERR_CUDA;
  }
  if (plan) {
    if (launch_scatter_plan(a, trunc, gb, s) != cudaSuccess) return GMI_ERR_CUDA;
  } else if (gb > 0) {
    bin_scatter_kernel<<<gb, 256, 0, s>>>(a);
    if (cudaGetLastError() != cudaSuccess) return GMI_ERR_CUDA;
  }
  profile_end(pb, s);
  return GMI_OK;
}

// Binning + plan + near + far on prepared arguments (single image or batch).
gmi_status run_forward_pipeline(KArgs& a, const WsLayout& L, void* ws, int mth, int mtw, bool trunc,
                                cudaStream_t s, int ppk) {
  if (ppk && !trunc) {
    // exact mode with per-point sigmas: the bins, then every micro-tile
    // through the per-pixel shifted gather (no plan, no near kernel)
    gmi_status st = run_bin_and_plan(a, L, ws, mth, mtw, trunc, s, false);
    if (st != GMI_OK) return st;
    const ProfileMark pf = profile_begin(GMI_STAGE_FAR, s);
    if (launch_pp_exact_forward(a, mth, mtw, ppk, s) != cudaSuccess) return GMI_ERR_CUDA;
    profile_end(pf, s);
    return GMI_OK;
  }
  gmi_status st = run_bin_and_plan(a, L, ws, mth, mtw, trunc, s, true);
  if (st != GMI_OK) return st;
  const int sms = device_sm_count();
  const bool staged = uses_staged_gather(a.gather, ppk);
  const int per_sm = staged ? staged_blocks_per_sm(mth, mtw, a.C, trunc) : near_blocks_per_sm(mth, mtw, a.C, trunc, ppk);
  // persistent: at most one resident wave, and no more warps than work items can use
  const int gn = (int)std::max<long long>(1, std::min<long long>(a.wt_total * 4, (long long)sms * per_sm));
  // Single images up to kFarInNearPixels: the near kernel's warps take the
  // far-field micro-tiles once their near work is done, which saves the far
  // launch (measured: 1024^2 upsampling 45.6 -> 44.4 us; a clustered 512^2
  // frame 85.5 -> 80.0 us).  Larger images and batches keep the far kernel,
  // whose fuller grid wins on large far fields (clustered 2048^2: 748 vs
  // 805 us; the 64-image batch: 1048 vs 1129 us).
  constexpr long long kFarInNearPixels = 1LL << 21;
  a.far_in_near =
      staged && !trunc && !a.totals && (long long)a.g0.H * a.g0.W <= kFarInNearPixels ? 1 : 0;
  a.stage_wait_polls = stage_wait_polls();
  const ProfileMark pn = profile_begin(GMI_STAGE_NEAR, s);
  const cudaError_t en = staged ? launch_near_staged(a, mth, mtw, trunc, gn, s) : launch_near(a, mth, mtw, trunc, ppk, gn, s);
  if (en != cudaSuccess) return GMI_ERR_CUDA;
  profile_end(pn, s);
  if (!trunc && !a.far_in_near) {
    const ProfileMark pf = profile_begin(GMI_STAGE_FAR, s);
    if (launch_far(a, mth, mtw, sms, s) != cudaSuccess) return GMI_ERR_CUDA;
    profile_end(pf, s);
  }
  return GMI_OK;
}

bool uses_staged_gather(int gather, int ppk) { return ppk == 0 && gather != GMI_GATHER_DIRECT; }

void warm_near_caches(int mth, int mtw, int C, bool trunc, int ppk, int gather) {
  device_sm_count();
  scan_one_capacity();
  if (ppk && !trunc) {
    warm_pp_exact(C, ppk);
    return;
  }
  warm_scatter_plan();
  if (uses_staged_gather(gather, ppk)) staged_blocks_per_sm(mth, mtw, C, trunc);
  else near_blocks_per_sm(mth, mtw, C, trunc, ppk);
}

void warm_forward_caches(int C, const gmi_params* p) {
  int mth, mtw;
  variant_dims(p->variant, &mth, &mtw);
  warm_near_caches(mth, mtw, C, p->mode == GMI_MODE_TRUNCATED, 0, p->gather);
}

gmi_status read_status(const void* ws, cudaStream_t s) {
  if (cudaStreamSynchronize(s) != cudaSuccess) return GMI_ERR_CUDA;
  unsigned st = 0;
  if (cudaMemcpy(&st, ws, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return GMI_ERR_CUDA;
  if (st & ST_NONFINITE) return GMI_ERR_NONFINITE;
  if (st & ST_SIGMA) return GMI_ERR_INVALID_ARG;
  if (st & (ST_INTERNAL | ST_BOUNDS | ST_CANARY)) return GMI_ERR_INTERNAL;
  if (st & (ST_TIMEOUT | ST_BINS)) return GMI_ERR_TIMEOUT;
  return GMI_OK;
}

}  // namespace gmi

using namespace gmi;

// Forward pass with one shared sigma (sigmas == null) or per-point sigmas,
// pp_kind floats per point: isotropic [N], axis-aligned [N,2] or full [N,3].
// fwd_share: the workspace need only hold the forward's leading part of the
// layout (everything before the backward's region), which the forward alone
// touches.
static gmi_status forward_impl(const float* points, const float* values, const float* sigmas, int pp_kind,
                               int64_t N, int C, int H, int W, const gmi_params* p, float* image, float* den_out,
                               float* shift_out, void* workspace, size_t ws_bytes, gmi_stream_t stream,
                               bool fwd_share = false) {
  gmi_status st = check_params(p);
  if (st != GMI_OK) return st;
  if ((st = check_shape(N, C, H, W)) != GMI_OK) return st;
  if (!image || (N > 0 && (!points || !values))) return GMI_ERR_INVALID_ARG;
  if (((uintptr_t)points & 7u) != 0 || ((uintptr_t)values & 3u) != 0 || ((uintptr_t)image & 3u) != 0)
    return GMI_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int mth, mtw;
  variant_dims(p->variant, &mth, &mtw);
  ImageGeom g;
  memset(&g, 0, sizeof(g));
  fill_geom(g, N, H, W, p->sigma, p->radius_sigmas, p->bin_px, mth, mtw);
  g.points = points;
  g.values = values;
  g.image = image;
  g.den = den_out;
  g.shift = shift_out;
  g.sigmas = sigmas;
  g.pp_kind = sigmas ? pp_kind : 0;
  set_vec_ok(g);
  const long long nb = (long long)g.nbx * g.nby;
  const long long mt = (long long)g.mtx * g.mty;
  const long long wt = (long long)g.wtx * g.wty;
  const WsLayout L =
      ws_layout(N, nb, mt, wt, sat_entries(g), slot_bytes_for(mth, mtw, C), bwd_extra_bytes(N, C, H, W), true);
  if (!workspace || ((uintptr_t)workspace & 255u) != 0 || ws_bytes < (fwd_share ? L.extra : L.total))
    return GMI_ERR_WORKSPACE;

  if (N == 0) {  // no known point: colour 0 and den 0 everywhere
    const size_t px = (size_t)H * (size_t)W;
    if (cudaMemsetAsync(image, 0, px * C * sizeof(float), s) != cudaSuccess) return GMI_ERR_CUDA;
    if (den_out && cudaMemsetAsync(den_out, 0, px * sizeof(float), s) != cudaSuccess) return GMI_ERR_CUDA;
    if (shift_out && cudaMemsetAsync(shift_out, 0, px * sizeof(float), s) != cudaSuccess) return GMI_ERR_CUDA;
    if (cudaMemsetAsync(workspace, 0, sizeof(unsigned) * kStatusWords, s) != cudaSuccess) return GMI_ERR_CUDA;
    if (kGuardBytes > 0) {   // checked builds: every guard written, as by any other call
      Guards gx = L.guards;
      if (!fwd_share) bwd_guards(N, C, H, W, L.extra, gx);
      if (launch_canaries(workspace, gx, false, (unsigned*)workspace, s) != cudaSuccess) return GMI_ERR_CUDA;
    }
    return (p->flags & GMI_FLAG_SYNC_CHECK) ? read_status(workspace, s) : GMI_OK;
  }

  KArgs a;
  memset(&a, 0, sizeof(a));
  a.w = bind_ws(workspace, L);
  a.g0 = g;
  a.n_images = 1;
  a.C = C;
  a.n_total = N;
  a.nb_total = nb;
  a.wt_total = wt;
  a.ch_total = (N + kChunk - 1) / kChunk;
  a.mt_total = mt;
  a.satj_total = sat_jobs(g);
  a.gather = p->gather;
  const bool trunc = p->mode == GMI_MODE_TRUNCATED;
  const int ppk = g.pp_kind == 3 ? 2 : (g.pp_kind ? 1 : 0);
  if (!uses_staged_gather(p->gather, ppk)) a.w.tplan = nullptr;   // the plan writes none
  if (kGuardBytes > 0 && !fwd_share) {
    // checked builds: the backward region's guards too, so that a check after
    // any full-size call finds every guard written
    Guards gx;
    gx.n = 0;
    bwd_guards(N, C, H, W, L.extra, gx);
    if (launch_canaries(workspace, gx, false, a.w.status, s) != cudaSuccess) return GMI_ERR_CUDA;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if ((p->flags & GMI_FLAG_GRAPH) && !profile_on() && cudaStreamIsCapturing(s, &cap) == cudaSuccess &&
      cap == cudaStreamCaptureStatusNone) {
    FwdGraphKey key;
    memset(&key, 0, sizeof(key));
    cudaGetDevice(&key.device);
    key.C = C;
    key.H = H;
    key.W = W;
    key.N = N;
    key.points = points;
    key.values = values;
    key.sigmas = sigmas;
    key.pp_kind = g.pp_kind;
    key.image = image;
    key.den = den_out;
    key.shift = shift_out;
    key.ws = workspace;
    key.ws_bytes = ws_bytes;
    key.params = *p;
    // fill the host-side caches the launch sequence reads before any capture starts
    warm_near_caches(mth, mtw, C, trunc, ppk, p->gather);
    struct Ctx {
      const KArgs* a;
      const WsLayout* L;
      void* ws;
      int mth, mtw;
      bool trunc;
      int ppk;
    } ctx{&a, &L, workspace, mth, mtw, trunc, ppk};
    auto launch = [](void* c, cudaStream_t cs) -> gmi_status {
      const Ctx* x = static_cast<const Ctx*>(c);
      KArgs ka = *x->a;
      return run_forward_pipeline(ka, *x->L, x->ws, x->mth, x->mtw, x->trunc, cs, x->ppk);
    };
    st = forward_graphed(key, launch, &ctx, s);
  } else {
    st = run_forward_pipeline(a, L, workspace, mth, mtw, trunc, s, ppk);
  }
  if (st != GMI_OK) return st;
  return (p->flags & GMI_FLAG_SYNC_CHECK) ? read_status(workspace, s) : GMI_OK;
}

namespace gmi {

gmi_status forward_share_bytes(int64_t N, int C, int H, int W, const gmi_params* p, size_t* bytes) {
  gmi_status st = check_params(p);
  if (st != GMI_OK) return st;
  if ((st = check_shape(N, C, H, W)) != GMI_OK) return st;
  int mth, mtw;
  variant_dims(p->variant, &mth, &mtw);
  ImageGeom g;
  memset(&g, 0, sizeof(g));
  fill_geom(g, N, H, W, p->sigma, p->radius_sigmas, p->bin_px, mth, mtw);
  const long long nb = (long long)g.nbx * g.nby;
  const long long mt = (long long)g.mtx * g.mty;
  const long long wt = (long long)g.wtx * g.wty;
  *bytes = ws_layout(N, nb, mt, wt, sat_entries(g), slot_bytes_for(mth, mtw, C), 0, true).extra;
  return GMI_OK;
}

gmi_status forward_in_share(const float* points, const float* values, int64_t N, int C, int H, int W,
                            const gmi_params* p, float* image, float* den_out, float* shift_out, void* workspace,
                            size_t ws_bytes, gmi_stream_t stream) {
  return forward_impl(points, values, nullptr, 0, N, C, H, W, p, image, den_out, shift_out, workspace, ws_bytes,
                      stream, true);
}

}  // namespace gmi

namespace gmi {

static std::atomic<long long> g_wait_polls{-1};

long long wait_polls_setting() { return g_wait_polls.load(); }

}  // namespace gmi

extern "C" gmi_status gmi_set_wait_polls(int64_t polls) {
  g_wait_polls.store((long long)polls);
  return GMI_OK;
}

extern "C" {

const char* gmi_version(void) { return "gmi 0.1.0 sm_103a"; }

const char* gmi_status_string(gmi_status s) {
  switch (s) {
    case GMI_OK: return "GMI_OK";
    case GMI_ERR_INVALID_ARG: return "GMI_ERR_INVALID_ARG";
    case GMI_ERR_NONFINITE: return "GMI_ERR_NONFINITE";
    case GMI_ERR_WORKSPACE: return "GMI_ERR_WORKSPACE";
    case GMI_ERR_CUDA: return "GMI_ERR_CUDA";
    case GMI_ERR_BUDGET: return "GMI_ERR_BUDGET";
    case GMI_ERR_TIMEOUT: return "GMI_ERR_TIMEOUT";
    case GMI_ERR_UNSUPPORTED: return "GMI_ERR_UNSUPPORTED";
    case GMI_ERR_NOT_FOUND: return "GMI_ERR_NOT_FOUND";
    case GMI_ERR_CAPACITY: return "GMI_ERR_CAPACITY";
    case GMI_ERR_INTERNAL: return "GMI_ERR_INTERNAL";
  }
  return "GMI_ERR_UNKNOWN";
}

gmi_status gmi_params_default(gmi_params* p) {
  if (!p) return GMI_ERR_INVALID_ARG;
  memset(p, 0, sizeof(*p));
  p->sigma = 1.0f;
  p->radius_sigmas = 6.0f;
  p->mode = GMI_MODE_EXACT;
  return GMI_OK;
}

gmi_status gmi_workspace_size(int64_t N, int C, int H, int W, const gmi_params* p, size_t* bytes) {
  if (!bytes) return GMI_ERR_INVALID_ARG;
  gmi_status st = check_params(p);
  if (st != GMI_OK) return st;
  if ((st = check_shape(N, C, H, W)) != GMI_OK) return st;
  int mth, mtw;
  variant_dims(p->variant, &mth, &mtw);
  ImageGeom g;
  memset(&g, 0, sizeof(g));
  fill_geom(g, N, H, W, p->sigma, p->radius_sigmas, p->bin_px, mth, mtw);
  const long long nb = (long long)g.nbx * g.nby;
  const long long mt = (long long)g.mtx * g.mty;
  const long long wt = (long long)g.wtx * g.wty;
  *bytes = ws_layout(N, nb, mt, wt, sat_entries(g), slot_bytes_for(mth, mtw, C), bwd_extra_bytes(N, C, H, W), true).total;
  return GMI_OK;
}

gmi_status gmi_workspace_layout(int64_t N, int C, int H, int W, const gmi_params* p, gmi_ws_layout* out) {
  if (!out) return GMI_ERR_INVALID_ARG;
  gmi_status st = check_params(p);
  if (st != GMI_OK) return st;
  if ((st = check_shape(N, C, H, W)) != GMI_OK) return st;
  int mth, mtw;
  variant_dims(p->variant, &mth, &mtw);
  ImageGeom g;
  memset(&g, 0, sizeof(g));
  fill_geom(g, N, H, W, p->sigma, p->radius_sigmas, p->bin_px, mth, mtw);
  const long long nb = (long long)g.nbx * g.nby;
  const long long mt = (long long)g.mtx * g.mty;
  const long long wt = (long long)g.wtx * g.wty;
  const WsLayout L = ws_layout(N, nb, mt, wt, sat_entries(g), slot_bytes_for(mth, mtw, C), bwd_extra_bytes(N, C, H, W), true);
  out->off = L.off;
  out->oob = L.oob;
  out->sxy = L.sxy;
  out->sval = L.sval;
  out->perm = L.perm;
  out->bin_px = g.b;
  out->nbx = g.nbx;
  out->nby = g.nby;
  out->total = L.total;
  out->ubound = L.ubound;
  out->mth = mth;
  out->mtw = mtw;
  out->wtx = g.wtx;
  out->wty = g.wty;
  out->sat = L.sat;
  return GMI_OK;
}

gmi_status gmi_forward(const float* points, const float* values, int64_t N, int C, int H, int W,
                       const gmi_params* p, float* image, float* den_out, float* shift_out,
                       void* workspace, size_t ws_bytes, gmi_stream_t stream) {
  return forward_impl(points, values, nullptr, 0, N, C, H, W, p, image, den_out, shift_out, workspace,
                      ws_bytes, stream);
}

static gmi_status forward_per_point(const float* points, const float* values, const float* sigmas, int pp_kind,
                                    int64_t N, int C, int H, int W, const gmi_params* p, float* image,
                                    float* den_out, void* workspace, size_t ws_bytes, gmi_stream_t stream) {
  gmi_status st = check_params(p);
  if (st != GMI_OK) return st;
  if (N > 0 && (!sigmas || ((uintptr_t)sigmas & 3u) != 0)) return GMI_ERR_INVALID_ARG;
  return forward_impl(points, values, N > 0 ? sigmas : nullptr, pp_kind, N, C, H, W, p, image, den_out, nullptr,
                      workspace, ws_bytes, stream);
}

gmi_status gmi_forward_pp(const float* points, const float* values, const float* sigmas, int64_t N, int C, int H,
                          int W, const gmi_params* p, float* image, float* den_out, void* workspace,
                          size_t ws_bytes, gmi_stream_t stream) {
  return forward_per_point(points, values, sigmas, 1, N, C, H, W, p, image, den_out, workspace, ws_bytes,
                           stream);
}

gmi_status gmi_forward_aniso(const float* points, const float* values, const float* sigmas_xy, int64_t N, int C,
                             int H, int W, const gmi_params* p, float* image, float* den_out, void* workspace,
                             size_t ws_bytes, gmi_stream_t stream) {
  return forward_per_point(points, values, sigmas_xy, 2, N, C, H, W, p, image, den_out, workspace, ws_bytes,
                           stream);
}

gmi_status gmi_forward_cov(const float* points, const float* values, const float* cov, int64_t N, int C, int H,
                           int W, const gmi_params* p, float* image, float* den_out, void* workspace,
                           size_t ws_bytes, gmi_stream_t stream) {
  return forward_per_point(points, values, cov, 3, N, C, H, W, p, image, den_out, workspace, ws_bytes, stream);
}

gmi_status gmi_workspace_status(const void* workspace, gmi_stream_t stream) {
  if (!workspace) return GMI_ERR_INVALID_ARG;
  return read_status(workspace, (cudaStream_t)stream);
}

}  // extern "C"
