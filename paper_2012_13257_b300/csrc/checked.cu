// Memory-safety checks of the checked build (compiled with -DGMI_CHECKED),
// in place of a sanitizer: guard areas after every workspace region, written
// with a known pattern at the start of each call and tested afterwards, and
// the status words the bounds checks of the kernels (GMI_IN_BOUNDS) set.
// Nothing here traps or faults: a failure is a status the host reads.  In
// other builds the entry points answer GMI_ERR_UNSUPPORTED.
#include <string.h>

#include "api_internal.h"

struct gmi_batch_plan;

namespace gmi {

// One block per guard area, one thread per word.
__global__ void __launch_bounds__(64) canary_kernel(char* ws, Guards g, int verify, unsigned* status) {
  const int k = blockIdx.x;
  if (k >= g.n) return;
  unsigned* w = reinterpret_cast<unsigned*>(ws + g.off[k]);
  for (int i = threadIdx.x; i < (int)(kGuardBytes / 4); i += blockDim.x) {
    const unsigned want = kCanary ^ (unsigned)i;
    if (!verify) {
      w[i] = want;
    } else if (w[i] != want) {
      atomicOr(&status[kStatusErr], ST_CANARY);
      atomicCAS(&status[kBadGuard], 0u, (unsigned)k + 1u);
    }
  }
}

cudaError_t launch_canaries(void* ws, const Guards& g, bool verify, unsigned* status, cudaStream_t s) {
  if (kGuardBytes == 0 || g.n == 0) return cudaSuccess;
  canary_kernel<<<g.n, 64, 0, s>>>((char*)ws, g, verify ? 1 : 0, status);
  return cudaGetLastError();
}

// Tests the guards, waits, and turns the status words into a result:
// report[0] status bits, [1] the first failed bounds check's site, [2] its
// index, [3] the first overwritten guard's number + 1.
static gmi_status verify(void* ws, const Guards& g, cudaStream_t s, uint32_t* report) {
  unsigned* status = reinterpret_cast<unsigned*>(ws);
  if (launch_canaries(ws, g, true, status, s) != cudaSuccess) return GMI_ERR_CUDA;
  unsigned words[kStatusWords];
  if (cudaMemcpyAsync(words, ws, sizeof(words), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return GMI_ERR_CUDA;
  if (report) {
    report[0] = words[kStatusErr];
    report[1] = words[kBadSite];
    report[2] = words[kBadIndex];
    report[3] = words[kBadGuard];
  }
  return (words[kStatusErr] & (ST_BOUNDS | ST_CANARY)) ? GMI_ERR_INTERNAL : GMI_OK;
}

// The workspace of the batched plan (batch.cu) and its layout.
void batch_plan_workspace(const gmi_batch_plan* p, void** base, const WsLayout** L);

}  // namespace gmi

using namespace gmi;

extern "C" gmi_status gmi_check_workspace(int64_t N, int C, int H, int W, const gmi_params* p, void* workspace,
                                          size_t ws_bytes, gmi_stream_t stream, uint32_t* report) {
  if (kGuardBytes == 0) return GMI_ERR_UNSUPPORTED;
  gmi_status st = check_params(p);
  if (st != GMI_OK) return st;
  if ((st = check_shape(N, C, H, W)) != GMI_OK) return st;
  if (!workspace || ((uintptr_t)workspace & 255u) != 0) return GMI_ERR_WORKSPACE;
  int mth, mtw;
  variant_dims(p->variant, &mth, &mtw);
  ImageGeom g;
  memset(&g, 0, sizeof(g));
  fill_geom(g, N, H, W, p->sigma, p->radius_sigmas, p->bin_px, mth, mtw);
  const long long nb = (long long)g.nbx * g.nby, mt = (long long)g.mtx * g.mty, wt = (long long)g.wtx * g.wty;
  const WsLayout L =
      ws_layout(N, nb, mt, wt, sat_entries(g), slot_bytes_for(mth, mtw, C), bwd_extra_bytes(N, C, H, W), true);
  if (ws_bytes < L.extra) return GMI_ERR_WORKSPACE;
  Guards gd = L.guards;
  if (ws_bytes >= L.total) bwd_guards(N, C, H, W, L.extra, gd);   // written by every full-size call
  return verify(workspace, gd, (cudaStream_t)stream, report);
}

extern "C" gmi_status gmi_batch_check_workspace(const gmi_batch_plan* plan, gmi_stream_t stream, uint32_t* report) {
  if (kGuardBytes == 0) return GMI_ERR_UNSUPPORTED;
  if (!plan) return GMI_ERR_INVALID_ARG;
  void* base = nullptr;
  const WsLayout* L = nullptr;
  batch_plan_workspace(plan, &base, &L);
  return verify(base, L->guards, (cudaStream_t)stream, report);
}

extern "C" int gmi_is_checked_build(void) { return kGuardBytes > 0 ? 1 : 0; }
