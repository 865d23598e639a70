// Point binning: a counting sort of the known points into square bins of
// b x b output pixels, so that the gather kernels can enumerate the points
// near any pixel block as a few contiguous row segments.  The paper's
// truncation ("consider only those known points that are close enough",
// section 2) is what makes spatial binning sufficient.
//
//   bin_count    key = (clamped bin row, bin column); rank = atomic slot in the
//                bin; flags non-finite positions, per-point sigmas out of range
//                and bins holding out-of-frame points
//   scan_partial per-block sums of the bin counts
//   scan_final   exclusive scan of the counts, in place, into bin offsets
//   bin_scatter  bin-sorted copies of positions (float2) and colours (float4);
//                flags non-finite colours
#include "bin_body.cuh"
#include "api_internal.h"

#include <algorithm>

namespace gmi {

// Per-point sigmas of one point: false when finite but out of range (sx, sy
// in [sigma 2^-32, sigma]; a full covariance also needs |rho| <= 0.99 and
// its largest eigenvalue <= sigma^2, so that its ellipse stays inside the
// k sigma search radius); clears fin when one is NaN or Inf.
static __device__ __forceinline__ bool sigmas_ok(const ImageGeom& g, const float* sg, bool& fin) {
  bool f = true;
  for (int e = 0; e < g.pp_kind; ++e) f = f && isfinite(sg[e]);
  if (!f) {
    fin = false;
    return true;
  }
  const float lo = g.sigma * 0x1p-32f;
  const float sy = g.pp_kind >= 2 ? sg[1] : sg[0];
  bool ok = sg[0] >= lo && sg[0] <= g.sigma && sy >= lo && sy <= g.sigma;
  if (g.pp_kind == 3) {
    const float a = sg[0] * sg[0], c = sy * sy, b = sg[2] * sg[0] * sy, h = 0.5f * (a - c);
    const float lam = 0.5f * (a + c) + sqrtf(fmaf(h, h, b * b));
    ok = ok && fabsf(sg[2]) <= 0.99f && lam <= g.sigma * g.sigma * (1.0f + 0x1p-20f);
  }
  return ok;
}

__global__ void __launch_bounds__(256) bin_count_kernel(KArgs a_in) {
  const KArgs a = resolve(a_in);
  unsigned bad = 0, bad_sigma = 0;
  for (long long ch = blockIdx.x; ch < a.ch_total; ch += gridDim.x) {
    const int img = find_image<0>(a, ch);
    const ImageGeom g = a.w.table ? a.w.table[img] : a.g0;   // a copy: no address of a local struct
    const long long i = (ch - g.ch_base) * kChunk + threadIdx.x;
    if (i < g.n) {
      float2 p = reinterpret_cast<const float2*>(g.points)[i];
      bool fin = isfinite(p.x) && isfinite(p.y);   // (the colours are checked by the scatter, which reads them)
      if (g.sigmas && !sigmas_ok(g, g.sigmas + g.pp_kind * i, fin)) bad_sigma = 1;
      if (!fin) bad = 1;
      long long bin;
      bool oob;
      point_bin(g, p.x, p.y, bin, oob);
      if (GMI_IN_BOUNDS(a.w, bin, a.nb_total, CK_BIN)) {
        a.w.rank[g.pt_base + i] = atomicAdd(&a.w.off[bin], 1u);
        if (oob) a.w.oob[bin] = 1;
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&a.w.status[kStatusErr], ST_NONFINITE);
  if (__any_sync(0xffffffffu, bad_sigma) && (threadIdx.x & 31) == 0) atomicOr(&a.w.status[kStatusErr], ST_SIGMA);
}

// Sum of kScanChunk consecutive counts per block.
__global__ void __launch_bounds__(256) scan_partial_kernel(const unsigned* __restrict__ cnt, long long nb,
                                                           unsigned* __restrict__ partials, const long long* totals) {
  __shared__ unsigned red[8];
  if (totals) nb = totals[kTotBins];
  const long long base = (long long)blockIdx.x * kScanChunk;
  // batched calls size the grid by the plan's capacity: blocks past the bins
  // leave at once (no later block reads their partial)
  if (base >= nb) return;
  unsigned s = 0;
  for (int k = threadIdx.x; k < kScanChunk; k += blockDim.x) {
    long long j = base + k;
    if (j < nb) s += cnt[j];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    partials[blockIdx.x] = t;
  }
}

// Exclusive scan of the counts into offsets (in place); off[nb] = total.
// Each block adds the sum of all earlier blocks' partials, then scans its own
// kScanChunk bins (kScanChunk / 256 consecutive bins per thread).
__global__ void __launch_bounds__(256) scan_final_kernel(unsigned* __restrict__ off, long long nb,
                                                         const unsigned* __restrict__ partials, const long long* totals) {
  constexpr int kPer = kScanChunk / 256;
  if (totals) nb = totals[kTotBins];
  // blocks past the bins (capacity-sized grids of batched calls) leave at
  // once, before summing their predecessors' partials; block 0 stays for nb = 0
  if ((long long)blockIdx.x * kScanChunk >= nb && blockIdx.x > 0) return;
  __shared__ unsigned warp_tot[8];
  __shared__ unsigned block_prefix;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  unsigned pre = 0;
  for (int k = tid; k < (int)blockIdx.x; k += blockDim.x) pre += partials[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) pre += __shfl_xor_sync(0xffffffffu, pre, o);
  if (lane == 0) warp_tot[wid] = pre;
  __syncthreads();
  if (tid == 0) {
    unsigned t = 0;
    for (int w = 0; w < 8; ++w) t += warp_tot[w];
    block_prefix = t;
  }
  __syncthreads();
  const unsigned bpre = block_prefix;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kScanChunk + (long long)tid * kPer;
  unsigned v[kPer];
  unsigned s = 0;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    long long j = base + k;
    v[k] = j < nb ? off[j] : 0u;
    s += v[k];
  }
  unsigned incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  unsigned wpre = 0;
  for (int w = 0; w < wid; ++w) wpre += warp_tot[w];
  unsigned run = bpre + wpre + incl - s;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    long long j = base + k;
    if (j < nb) off[j] = run;
    run += v[k];
  }
  // the thread owning the last bin also writes the total into off[nb]
  if (nb > 0 && base <= nb - 1 && nb - 1 < base + kPer) off[nb] = run;
  if (nb == 0 && blockIdx.x == 0 && tid == 0) off[0] = 0;
}


// The same exclusive scan in one launch, for grids that are resident all at
// once (launched cooperatively, so the hardware guarantees it): each block
// sums its chunk and publishes the sum, waits at a grid barrier until every
// block has, then adds the sums of the earlier chunks to its own scan.  The
// wait is bounded (`polls` polls, at most kScanWaitPolls, about 0.1 s); a
// block that gives up sets ST_TIMEOUT and ST_BINS and goes on: its offsets
// are then wrong, so the scatter keeps every write inside its arrays, the
// plan marks every micro-tile inactive and queues no far-field work, the
// other kernels that follow the offsets leave at once (bins_invalid), and the
// call reports the timeout.
constexpr unsigned kScanWaitPolls = 1u << 20;

unsigned scan_wait_polls() {
  const long long v = wait_polls_setting();
  return v < 0 ? kScanWaitPolls : (unsigned)std::min<long long>(v, (long long)kScanWaitPolls);
}

__global__ void __launch_bounds__(256) scan_one_kernel(unsigned* __restrict__ off, long long nb,
                                                       unsigned* __restrict__ partials, unsigned* status,
                                                       unsigned polls) {
  constexpr int kPer = kScanChunk / 256;
  __shared__ unsigned warp_tot[8];
  __shared__ unsigned block_prefix;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const long long base = (long long)blockIdx.x * kScanChunk + (long long)tid * kPer;
  unsigned v[kPer];
  unsigned s = 0;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    v[k] = base + k < nb ? off[base + k] : 0u;
    s += v[k];
  }
  unsigned incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  unsigned wpre = 0, btot = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    if (w < wid) wpre += warp_tot[w];
    btot += warp_tot[w];
  }
  // publish this chunk's sum, then wait for every block's
  if (tid == 0) {
    partials[blockIdx.x] = btot;
    __threadfence();
    atomicAdd(&status[kScanArrive], 1u);
    for (unsigned k = 0;; ++k) {
      if (k >= polls) {
        atomicOr(&status[kStatusErr], ST_TIMEOUT | ST_BINS);
        break;
      }
      unsigned n;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(n) : "l"(status + kScanArrive) : "memory");
      if (n >= gridDim.x) break;
      __nanosleep(64);
    }
  }
  __syncthreads();
  // the sums of the earlier chunks
  unsigned pre = 0;
  for (int k = tid; k < (int)blockIdx.x; k += blockDim.x) pre += __ldcg(&partials[k]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) pre += __shfl_xor_sync(0xffffffffu, pre, o);
  __syncthreads();   // warp_tot is free again
  if (lane == 0) warp_tot[wid] = pre;
  __syncthreads();
  if (tid == 0) {
    unsigned t = 0;
    for (int w = 0; w < 8; ++w) t += warp_tot[w];
    block_prefix = t;
  }
  __syncthreads();
  unsigned run = block_prefix + wpre + incl - s;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    if (base + k < nb) off[base + k] = run;
    run += v[k];
  }
  if (nb > 0 && base <= nb - 1 && nb - 1 < base + kPer) off[nb] = run;
}

__global__ void __launch_bounds__(256) bin_scatter_kernel(KArgs a_in) {
  const KArgs a = resolve(a_in);
  if (bins_invalid(a.w.status)) return;
  bin_scatter_body(a, gridDim.x, blockIdx.x);
}

}  // namespace gmi

namespace gmi {

// Clears what a batched call needs at zero (sizes from the device totals).
__global__ void __launch_bounds__(256) batch_clear_kernel(KArgs a_in) {
  const KArgs a = resolve(a_in);
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (long long i = t0; i < kStatusWords; i += stride) a.w.status[i] = 0u;
  for (long long i = t0; i <= a.nb_total; i += stride) a.w.off[i] = 0u;
  for (long long i = t0; i < a.nb_total; i += stride) a.w.oob[i] = 0;
  for (long long i = t0; i < a.wt_total; i += stride) a.w.tile_done[i] = 0u;
  if (a.w.fbflag)
    for (long long i = t0; i < a.mt_total; i += stride) a.w.fbflag[i] = 0u;
}

}  // namespace gmi
