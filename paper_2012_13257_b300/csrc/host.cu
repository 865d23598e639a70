// gmi_forward_host: the forward pass end to end from host memory.  Two
// uploads into device copies held in the workspace, the forward pipeline of
// gmi_forward on them (in the forward's share of the workspace layout), and
// one download of the image, in order on the caller's stream; with
// GMI_FLAG_GRAPH and pinned host buffers the whole sequence is one cached
// CUDA graph.
#include <string.h>

#include "api_internal.h"

namespace {

size_t al256(size_t v) { return (v + 255) / 256 * 256; }

// [forward's share | points N x 2 | values N x C | image H x W x C], bytes
struct HostLayout {
  size_t fwd, pts, vals, img, total;
};

gmi_status host_layout(int64_t N, int C, int H, int W, const gmi_params* p, HostLayout* L) {
  size_t fwd = 0;
  const gmi_status st = gmi::forward_share_bytes(N, C, H, W, p, &fwd);
  if (st != GMI_OK) return st;
  L->fwd = al256(fwd);
  L->pts = L->fwd;
  L->vals = L->pts + al256(sizeof(float) * 2 * (size_t)N);
  L->img = L->vals + al256(sizeof(float) * (size_t)C * (size_t)N);
  L->total = L->img + al256(sizeof(float) * (size_t)C * (size_t)H * (size_t)W);
  return GMI_OK;
}

bool pinned(const void* ptr) {
  if (!ptr) return true;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

struct HostCall {
  const float *hp, *hv;
  float* hi;
  float *dp, *dv, *di;
  int64_t N;
  int C, H, W;
  gmi_params p;   // flags without GRAPH and SYNC_CHECK (the caller handles both)
  void* ws;
  size_t fwd_bytes;
};

gmi_status run_host(const HostCall& c, cudaStream_t s) {
  const size_t bp = sizeof(float) * 2 * (size_t)c.N, bv = sizeof(float) * (size_t)c.C * (size_t)c.N;
  const size_t bi = sizeof(float) * (size_t)c.C * (size_t)c.H * (size_t)c.W;
  if (bp && cudaMemcpyAsync(c.dp, c.hp, bp, cudaMemcpyHostToDevice, s) != cudaSuccess) return GMI_ERR_CUDA;
  if (bv && cudaMemcpyAsync(c.dv, c.hv, bv, cudaMemcpyHostToDevice, s) != cudaSuccess) return GMI_ERR_CUDA;
  const gmi_status st = gmi::forward_in_share(c.dp, c.dv, c.N, c.C, c.H, c.W, &c.p, c.di, nullptr, nullptr, c.ws,
                                              c.fwd_bytes, (gmi_stream_t)s);
  if (st != GMI_OK) return st;
  if (cudaMemcpyAsync(c.hi, c.di, bi, cudaMemcpyDeviceToHost, s) != cudaSuccess) return GMI_ERR_CUDA;
  return GMI_OK;
}

}  // namespace

extern "C" gmi_status gmi_forward_host_workspace_size(int64_t N, int C, int H, int W, const gmi_params* p,
                                                      size_t* bytes) {
  if (!bytes) return GMI_ERR_INVALID_ARG;
  HostLayout L;
  const gmi_status st = host_layout(N, C, H, W, p, &L);
  if (st != GMI_OK) return st;
  *bytes = L.total;
  return GMI_OK;
}

extern "C" gmi_status gmi_forward_host(const float* points_host, const float* values_host, int64_t N, int C,
                                       int H, int W, const gmi_params* p, float* image_host, void* workspace,
                                       size_t ws_bytes, gmi_stream_t stream) {
  HostLayout L;
  gmi_status st = host_layout(N, C, H, W, p, &L);
  if (st != GMI_OK) return st;
  if (!image_host || (N > 0 && (!points_host || !values_host))) return GMI_ERR_INVALID_ARG;
  if (((uintptr_t)points_host & 7u) != 0 || ((uintptr_t)values_host & 3u) != 0 || ((uintptr_t)image_host & 3u) != 0)
    return GMI_ERR_INVALID_ARG;
  if (!workspace || ((uintptr_t)workspace & 255u) != 0 || ws_bytes < L.total) return GMI_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  char* b = (char*)workspace;
  HostCall c{points_host, values_host, image_host, (float*)(b + L.pts), (float*)(b + L.vals), (float*)(b + L.img),
             N, C, H, W, *p, workspace, L.fwd};
  c.p.flags &= ~(GMI_FLAG_GRAPH | GMI_FLAG_SYNC_CHECK);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if ((p->flags & GMI_FLAG_GRAPH) && !gmi::profile_on() && cudaStreamIsCapturing(s, &cap) == cudaSuccess &&
      cap == cudaStreamCaptureStatusNone && pinned(points_host) && pinned(values_host) && pinned(image_host)) {
    gmi::FwdGraphKey key;
    memset(&key, 0, sizeof(key));
    cudaGetDevice(&key.device);
    key.C = C;
    key.H = H;
    key.W = W;
    key.N = N;
    key.points = points_host;
    key.values = values_host;
    key.image = image_host;
    key.ws = workspace;
    key.ws_bytes = ws_bytes;
    key.host = 1;
    key.params = *p;
    gmi::warm_forward_caches(C, p);
    auto launch = [](void* ctx, cudaStream_t cs) -> gmi_status { return run_host(*static_cast<HostCall*>(ctx), cs); };
    st = gmi::forward_graphed(key, launch, &c, s);
  } else {
    st = run_host(c, s);
  }
  if (st != GMI_OK) return st;
  return (p->flags & GMI_FLAG_SYNC_CHECK) ? gmi::read_status(workspace, s) : GMI_OK;
}
