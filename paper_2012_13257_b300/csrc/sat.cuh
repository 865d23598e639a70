// Summed-area table of the point bins (per image, (nby+1) x (nbx+1) counts:
// entry (by, bx) = points in bins [0, by) x [0, bx)), so that the far-field
// search counts any window of bins with four loads instead of two per bin
// row.  Built from the scanned bin offsets, column by column, by near-kernel
// warps that have run out of work, and only when the far-field queue is not
// empty; read by the far-field work that follows in the same kernel (after
// sat_wait) or in the far kernel.
#pragma once

#include "common.cuh"

namespace gmi {

// Claims 32-column jobs from status[kSatHead] until none is left; one warp,
// lane = column.  A column's entries are the running sums, down the bin rows,
// of that row's points in bins [0, bx) (off[row + bx] - off[row]).
static __device__ void sat_build(const KArgs& a) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned j = 0;
    if (lane == 0) j = atomicAdd(&a.w.status[kSatHead], 1u);
    j = __shfl_sync(full, j, 0);
    if ((long long)j >= a.satj_total) return;
    const int img = find_image<4>(a, (long long)j);
    const ImageGeom g = a.w.table ? a.w.table[img] : a.g0;   // a copy: no address of a local struct
    const int c = (int)((long long)j - g.satj_base) * 32 + lane;
    if (c <= g.nbx) {
      const unsigned* __restrict__ off = a.w.off + g.bin_base;
      unsigned* __restrict__ S = a.w.sat + g.sat_base;
      const long long st = g.nbx + 1;
      unsigned run = 0;
      S[c] = 0;
#pragma unroll 8
      for (int r = 0; r < g.nby; ++r) {
        const long long rs = (long long)r * g.nbx;
        run += __ldg(&off[rs + c]) - __ldg(&off[rs]);
        S[(long long)(r + 1) * st + c] = run;
      }
    }
    // the job's columns are visible device-wide before it counts as done
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicAdd(&a.w.status[kSatDone], 1u);
  }
}

// Waits (bounded: about 0.1 s) until every column job of the table is done;
// false, with ST_TIMEOUT set, if it gave up.  Every lane reads the counter
// with acquire semantics, so its later loads of the table see the entries.
constexpr unsigned kSatWaitPolls = 1u << 20;

static __device__ bool sat_wait(const KArgs& a) {
  for (unsigned k = 0; k < kSatWaitPolls; ++k) {
    unsigned n;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(n) : "l"(a.w.status + kSatDone) : "memory");
    if ((long long)n >= a.satj_total) return true;
    __nanosleep(64);
  }
  if ((threadIdx.x & 31) == 0) atomicOr(&a.w.status[kStatusErr], ST_TIMEOUT);
  return false;
}

// Points in the bins [bx_lo, bx_hi] x [by_lo, by_hi] of image g.
static __device__ __forceinline__ unsigned sat_count(const KArgs& a, const ImageGeom& g, int bx_lo, int bx_hi,
                                                     int by_lo, int by_hi) {
  const unsigned* __restrict__ S = a.w.sat + g.sat_base;
  const long long st = g.nbx + 1;
  const long long y0 = (long long)by_lo * st, y1 = (long long)(by_hi + 1) * st;
  // (coherent loads: the table may have been written earlier in the same kernel)
  return __ldcg(&S[y1 + bx_hi + 1]) - __ldcg(&S[y0 + bx_hi + 1]) - __ldcg(&S[y1 + bx_lo]) + __ldcg(&S[y0 + bx_lo]);
}

}  // namespace gmi
