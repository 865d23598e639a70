// Host-side helpers shared by the libgmi translation units.
#pragma once

#include <algorithm>

#include "common.cuh"
#include "gmi.h"

namespace gmi {

// Checked builds (-DGMI_CHECKED) leave a guard area of kGuardBytes after
// every workspace region, filled with kCanary at the start of each call and
// verified by gmi_check_workspace: a kernel writing past its region shows up
// there.  Other builds leave no guards.
#ifdef GMI_CHECKED
constexpr size_t kGuardBytes = 256;
#else
constexpr size_t kGuardBytes = 0;
#endif
constexpr unsigned kCanary = 0xC0DEFACEu;
constexpr int kMaxGuards = 24;
struct Guards {
  int n;
  size_t off[kMaxGuards];   // byte offsets of the guard areas from the workspace start
};

// Byte offsets of the regions of a workspace.
struct WsLayout {
  size_t status, off, oob, tile_done, zero_end, rank, sxy, sval, perm, spp, partials, farq, items, slots, ubound, sat,
      tplan, extra, total;
  bool has_tplan;
  unsigned cap_items, cap_slots;
  Guards guards;   // after every region (checked builds); the first four follow the cleared regions
};

// Checked builds: writes (verify = false) or tests (verify = true, ST_CANARY
// and the first bad guard's number + 1 in status[kBadGuard]) the guard areas.
cudaError_t launch_canaries(void* ws, const Guards& g, bool verify, unsigned* status, cudaStream_t s);

int device_sm_count();
void variant_dims(int variant, int* mth, int* mtw);
int auto_bin_px(long long n, int H, int W);
gmi_status check_params(const gmi_params* p);
gmi_status check_shape(long long N, int C, int H, int W);
void fill_geom(ImageGeom& g, long long N, int H, int W, float sigma, float k, int bin_px, int mth, int mtw);
void set_vec_ok(ImageGeom& g);
bool aligned16(const void* p);
size_t slot_bytes_for(int mth, int mtw, int C);
WsLayout ws_layout(long long n_total, long long nb_total, long long mt_total, long long wt_total,
                   long long sat_entries, size_t slot_bytes, long long extra_bytes, bool tile_plans = false);
// Summed-area table of one image's bins: entries and 32-column build jobs.
long long sat_entries(const ImageGeom& g);
long long sat_jobs(const ImageGeom& g);
DevWork bind_ws(void* ws, const WsLayout& L);
// gmi_set_wait_polls: the process-wide poll limit of the device waits that
// may be made to give up (negative: their defaults), and each wait's limit
// from it: the staged gather's first wait on its copies, the one-launch
// scan's grid barrier.
long long wait_polls_setting();
unsigned stage_wait_polls();
unsigned scan_wait_polls();

gmi_status run_bin_and_plan(KArgs& a, const WsLayout& L, void* ws, int mth, int mtw, bool trunc,
                            cudaStream_t s, bool plan);
// ppk: per-point sigmas (a.g0.sigmas set; truncated mode): 1 separable
// (isotropic or axis-aligned), 2 full covariance; 0 without
gmi_status run_forward_pipeline(KArgs& a, const WsLayout& L, void* ws, int mth, int mtw, bool trunc,
                                cudaStream_t s, int ppk = 0);
gmi_status read_status(const void* ws, cudaStream_t s);
// Fills the host-side caches a forward launch sequence reads (SM count,
// near-kernel occupancy), so that none is first computed inside a capture.
void warm_forward_caches(int C, const gmi_params* p);
// Whether a forward uses the staged near-field gather, given params->gather and the
// per-point kind (per-point sigmas use the direct gather).
bool uses_staged_gather(int gather, int ppk);
// Fills the SM-count and occupancy caches of the near kernel a call will launch.
void warm_near_caches(int mth, int mtw, int C, bool trunc, int ppk, int gather);

// Stage timing (profile.cu): no-ops unless gmi_profile_enable(1) was called.
// Every stage is also an NVTX range on the host thread that enqueues it
// ("gmi.bin", "gmi.near", "gmi.far", "gmi.backward"), for ncu --nvtx filters
// and timeline tools; without a tool attached the ranges cost nothing.
struct ProfileMark {
  int stage;
  cudaEvent_t a, b;
  bool range;   // an NVTX range was pushed
};
bool profile_on();
ProfileMark profile_begin(int stage, cudaStream_t s);
void profile_end(const ProfileMark& m, cudaStream_t s);

// Everything a single-image forward launch sequence depends on: the key of a
// cached graph (graph_cache.cu).  Built from a zeroed struct so that it
// compares bytewise.
struct FwdGraphKey {
  int device;
  int C, H, W;
  long long N;
  const void *points, *values, *sigmas, *image, *den, *shift, *ws;
  int pp_kind;
  int host;   // gmi_forward_host: points/values/image are host buffers, copies captured too
  size_t ws_bytes;
  gmi_params params;
};

// Launches the sequence `launch(ctx, stream)` records as a graph: replays the
// cached graph for `key`, or captures, instantiates, caches and launches one.
gmi_status forward_graphed(const FwdGraphKey& key, gmi_status (*launch)(void*, cudaStream_t), void* ctx,
                           cudaStream_t s);

// The forward's leading share of the workspace layout (the backward's region
// excluded), and a forward pass that needs only that share (no-alloc path).
gmi_status forward_share_bytes(int64_t N, int C, int H, int W, const gmi_params* p, size_t* bytes);
gmi_status forward_in_share(const float* points, const float* values, int64_t N, int C, int H, int W,
                            const gmi_params* p, float* image, float* den_out, float* shift_out, void* workspace,
                            size_t ws_bytes, gmi_stream_t stream);

// Extra workspace bytes the backward pass needs beyond the forward layout,
// and where its regions start inside the extra block.
long long bwd_extra_bytes(long long N, int C, int H, int W);
void bind_bwd(DevWork& w, void* extra, long long N, int C, int H, int W, long long mt_total);
// The guard areas of the backward's region (checked builds), appended to g
// with offsets from the workspace start (extra_at: where the region starts).
void bwd_guards(long long N, int C, int H, int W, size_t extra_at, Guards& g);

}  // namespace gmi
