// Candidate collection around a micro-tile, shared by the far-field forward
// kernel and the backward fallback kernel: Chebyshev windows over the bin
// grid, counted or enumerated one warp at a time.
#pragma once

#include "common.cuh"

namespace gmi {

constexpr int kFarCap = 1024;   // candidate indices per warp per chunk
constexpr int kFarWarps = 4;

struct FarTile {
  float xa, xb, ya, yb;   // pixel-centre rectangle of the micro-tile
};

__device__ __forceinline__ void window_bins(const ImageGeom& g, const FarTile& t, float h, int& bx_lo,
                                            int& bx_hi, int& by_lo, int& by_hi) {
  bx_lo = bin_coord(t.xa - h, g.inv_b, g.nbx);
  bx_hi = bin_coord(t.xb + h, g.inv_b, g.nbx);
  by_lo = bin_coord(t.ya - h, g.inv_b, g.nby);
  by_hi = bin_coord(t.yb + h, g.inv_b, g.nby);
}

// Number of points in the bins covering the Chebyshev window of half-width h.
static __device__ unsigned window_count(const KArgs& a, const ImageGeom& g, const FarTile& t, float h) {
  int bx_lo, bx_hi, by_lo, by_hi;
  window_bins(g, t, h, bx_lo, bx_hi, by_lo, by_hi);
  const int lane = threadIdx.x & 31;
  unsigned s = 0;
  for (int by = by_lo + lane; by <= by_hi; by += 32) {
    const long long rowb = g.bin_base + (long long)by * g.nbx;
    s += a.w.off[rowb + bx_hi + 1] - a.w.off[rowb + bx_lo];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Appends to L the indices of the points of the Chebyshev window of
// half-width h whose squared Euclidean distance to the pixel rectangle is at
// most r2 (r2 < 0: no filter), numbered [skip, skip + kFarCap) in enumeration
// order.  Returns how many points pass the filter in total.
static __device__ unsigned collect(const KArgs& a, const ImageGeom& g, const FarTile& t, float h, float r2,
                            unsigned skip, unsigned* L) {
  int bx_lo, bx_hi, by_lo, by_hi;
  window_bins(g, t, h, bx_lo, bx_hi, by_lo, by_hi);
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  unsigned total = 0;
  for (int by0 = by_lo; by0 <= by_hi; by0 += 32) {
    const int myrow = by0 + lane;
    unsigned s = 0, e = 0;
    if (myrow <= by_hi) {
      const long long rowb = g.bin_base + (long long)myrow * g.nbx;
      s = a.w.off[rowb + bx_lo];
      e = a.w.off[rowb + bx_hi + 1];
    }
    const int nrows = min(32, by_hi - by0 + 1);
    for (int r = 0; r < nrows; ++r) {
      const unsigned rs = __shfl_sync(full, s, r);
      const unsigned re = __shfl_sync(full, e, r);
      for (unsigned base = rs; base < re; base += 32) {
        const unsigned idx = base + lane;
        bool pass = false;
        if (idx < re) {
          if (r2 < 0.0f) {
            pass = true;
          } else {
            const float2 p = a.w.sxy[idx];
            const float dx = fmaxf(fmaxf(t.xa - p.x, p.x - t.xb), 0.0f);
            const float dy = fmaxf(fmaxf(t.ya - p.y, p.y - t.yb), 0.0f);
            pass = dx * dx + dy * dy <= r2;
          }
        }
        const unsigned m = __ballot_sync(full, pass);
        const unsigned pos = total + __popc(m & ((1u << lane) - 1u));
        if (pass && pos >= skip && pos < skip + kFarCap) L[pos - skip] = idx;
        total += __popc(m);
      }
    }
  }
  __syncwarp();
  return total;
}

}  // namespace gmi
