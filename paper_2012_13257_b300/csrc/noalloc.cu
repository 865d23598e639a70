// gmi_forward_noalloc: the forward pass for callers that cannot allocate
// device memory (host applications that own the GPU memory pool, loops that
// must not stall on cudaMalloc/cudaFree, bindings that cannot pass a
// workspace).  Its scratch is one statically sized device array compiled into
// this library; the pipeline it runs is gmi_forward's, unchanged, in the
// forward's share of the workspace layout (the backward's region left out).
#include "api_internal.h"

namespace {

constexpr size_t kScratchBytes = GMI_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The scratch array.  Its name is only a host-side stand-in in host code; the
// device address is looked up below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of the scratch array on the current device, looked up on
// every call with that device current: the lookup allocates nothing and is
// cheap, and an address kept from an earlier call could be stale after the
// device's context was reset and the module loaded again.  The first call on a
// device loads the module's symbols, so it should come before any stream
// capture.
gmi_status scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return GMI_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return GMI_ERR_UNSUPPORTED;
  void* a = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&a, g_scratch);
  if (e != cudaSuccess || a == nullptr) return GMI_ERR_CUDA;
  *out = a;
  return GMI_OK;
}

}  // namespace

extern "C" gmi_status gmi_forward_noalloc(const float* points, const float* values, int64_t N, int C, int H,
                                          int W, const gmi_params* p, float* image, float* den_out,
                                          float* shift_out, gmi_stream_t stream) {
  size_t need = 0;   // the forward's share of the workspace: it never touches the backward's region
  gmi_status st = gmi::forward_share_bytes(N, C, H, W, p, &need);
  if (st != GMI_OK) return st;
  if (need > kScratchBytes) return GMI_ERR_CAPACITY;   // too large for the static scratch
  void* ws = nullptr;
  if ((st = scratch_address(&ws)) != GMI_OK) return st;
  return gmi::forward_in_share(points, values, N, C, H, W, p, image, den_out, shift_out, ws, kScratchBytes, stream);
}
