// Far-field gather: exact Eq. 1 / Eq. 2 for micro-tiles that the near kernel
// could not take (pixels far from every known point, where the unshifted
// weights 2^(-kappa d^2) would underflow), one warp per queued micro-tile
// (far_entry in far_tile.cuh).  With the staged near kernel the same work runs
// in the near kernel's warps once their near work is done, and this kernel is
// not launched; the direct-load near kernel leaves it to this kernel.
#include "far_tile.cuh"

namespace gmi {

template <int C>
__global__ void __launch_bounds__(32 * kFarWarps) far_kernel(KArgs a_in, int mth, int mtw) {
  const KArgs a = resolve(a_in);
  if (bins_invalid(a.w.status)) return;
  __shared__ unsigned lists[kFarWarps][kFarCap];
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned* L = lists[wid];
  const unsigned nfar = a.w.status[kFarCount];

  // first entry by warp index, later ones claimed from the queue; with an
  // empty queue (the usual case for dense inputs) warps leave at once
  const unsigned n_warps = gridDim.x * kFarWarps;
  unsigned e = blockIdx.x * kFarWarps + wid;
  while (e < nfar) {
    far_entry<C>(a, mth, mtw, a.w.farq[e], L);
    __syncwarp();   // the candidate list is rewritten by the next entry
    unsigned ne = 0;
    if (lane == 0) ne = n_warps + atomicAdd(&a.w.status[kFarHead], 1u);
    e = __shfl_sync(full, ne, 0);
  }
}

// Resident far-kernel blocks per SM for C channels (cached).
static int far_blocks_per_sm(int C) {
  static int cache[kMaxC + 1];
  const int c = C < 1 ? 1 : (C > kMaxC ? kMaxC : C);
  if (cache[c] == 0) {
    int n = 0;
    switch (c) {
      case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, far_kernel<1>, 32 * kFarWarps, 0); break;
      case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, far_kernel<2>, 32 * kFarWarps, 0); break;
      case 3: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, far_kernel<3>, 32 * kFarWarps, 0); break;
      default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, far_kernel<4>, 32 * kFarWarps, 0); break;
    }
    cache[c] = n > 0 ? n : 1;
  }
  return cache[c];
}

// Persistent launch: every resident warp slot (the work is latency-bound).
cudaError_t launch_far(const KArgs& a, int mth, int mtw, int sms, cudaStream_t s) {
  const int grid = sms * far_blocks_per_sm(a.C);
  switch (a.C) {
    case 1: far_kernel<1><<<grid, 32 * kFarWarps, 0, s>>>(a, mth, mtw); break;
    case 2: far_kernel<2><<<grid, 32 * kFarWarps, 0, s>>>(a, mth, mtw); break;
    case 3: far_kernel<3><<<grid, 32 * kFarWarps, 0, s>>>(a, mth, mtw); break;
    default: far_kernel<4><<<grid, 32 * kFarWarps, 0, s>>>(a, mth, mtw); break;
  }
  return cudaGetLastError();
}

}  // namespace gmi
