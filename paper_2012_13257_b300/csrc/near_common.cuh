// Candidate windows of the near-field gather: the pixel-centre rectangle of
// one thread's micro-tile, its squared radius, and the bin-row segments of
// the bin-sorted point arrays that can hold a point within that radius.
// Shared by the plan, the direct-load gather and the staged gather.
#pragma once

#include "common.cuh"

#include <climits>

namespace gmi {

// Candidates one warp of the staged gather can stage at once, by micro-tile
// shape: the window of a 32 x 16 px warp tile (4 x 4 micro-tiles) at one
// point per bin and a 6.4 px radius is about 300 records in 14 bin rows.
template <int MTH, int MTW>
struct StageCap {
  static constexpr int value = MTH * MTW >= 16 ? 352 : 224;
};

__device__ __forceinline__ int warp_min(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ float warp_maxf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Candidate window of one thread: pixel-centre rectangle and radius.
struct LaneWin {
  float xq0, xq1, yq0, yq1;  // first / last pixel centres of the micro-tile
  float R2;                  // squared radius
  int by_lo, by_hi;          // bin rows that can hold a point within the radius
};

__device__ __forceinline__ LaneWin lane_window(const ImageGeom& g, int x0, int y0, int nx, int ny, float R2) {
  LaneWin w;
  w.xq0 = (float)x0 + 0.5f;
  w.yq0 = (float)y0 + 0.5f;
  w.xq1 = w.xq0 + (float)(nx - 1);
  w.yq1 = w.yq0 + (float)(ny - 1);
  w.R2 = R2;
  const float R = sqrtf(R2);
  w.by_lo = bin_coord(w.yq0 - R, g.inv_b, g.nby);
  w.by_hi = bin_coord(w.yq1 + R, g.inv_b, g.nby);
  return w;
}

// Bin columns [bx_lo, bx_hi] of bin row `by` that can hold a point within the
// radius of the window's pixels: the row's y-distance to the pixel rows
// narrows its x-extent hx (border rows can hold clamped out-of-frame points,
// so they get the full radius).  Monotone in the window: a window inside
// another (pixel rectangle and radius) gets a sub-range of its columns.
__device__ __forceinline__ void row_bins(const ImageGeom& g, const LaneWin& w, int by, int& bx_lo, int& bx_hi,
                                         float& hx) {
  const float bf = (float)g.b;
  float dyr = 0.0f;
  if (by > 0 && by < g.nby - 1) dyr = fmaxf(fmaxf((float)by * bf - w.yq1, w.yq0 - (float)(by + 1) * bf), 0.0f);
  hx = sqrtf(fmaxf(w.R2 - dyr * dyr, 0.0f));
  bx_lo = bin_coord(w.xq0 - hx, g.inv_b, g.nbx);
  bx_hi = bin_coord(w.xq1 + hx, g.inv_b, g.nbx);
}

// Sorted-array segment [s, e) of bin row `by` that can hold a point within
// the radius of the window's pixels (the points of its row_bins columns).
__device__ __forceinline__ void row_segment(const KArgs& a, const ImageGeom& g, const LaneWin& w, int by,
                                            unsigned& s, unsigned& e) {
  int bx_lo, bx_hi;
  float hx;
  row_bins(g, w, by, bx_lo, bx_hi, hx);
  const long long rowb = g.bin_base + (long long)by * g.nbx;
  s = __ldg(&a.w.off[rowb + bx_lo]);
  e = __ldg(&a.w.off[rowb + bx_hi + 1]);
}

// This work item's share [lo, hi) of the thread's candidate sequence (its
// window's row segments in order): item `split` of S takes the split-th of
// S nearly equal parts; S = 1 takes everything.
__device__ __forceinline__ void item_share(const KArgs& a, const ImageGeom& g, const LaneWin& w, unsigned split,
                                           unsigned S, unsigned& lo, unsigned& hi) {
  lo = 0u;
  hi = 0xffffffffu;
  if (S > 1) {
    unsigned n = 0;
    for (int yb = w.by_lo; yb <= w.by_hi; ++yb) {
      unsigned s0, e0;
      row_segment(a, g, w, yb, s0, e0);
      n += e0 - s0;
    }
    lo = (unsigned)(((unsigned long long)n * split) / S);
    hi = (unsigned)(((unsigned long long)n * (split + 1)) / S);
  }
}

// Walks the candidates [lo, hi) of the thread's window straight from the
// bin-sorted arrays in global memory (through L1), bin row by bin row, the
// next candidate and the next row's bounds always loaded one step ahead, and
// hands each to consume(position, colour, per-point constants).
template <bool PP, typename F>
__device__ __forceinline__ void direct_walk(const KArgs& a, const ImageGeom& g, const LaneWin& w, unsigned lo,
                                            unsigned hi, F& consume) {
  const float2* __restrict__ sxy = a.w.sxy;
  const float4* __restrict__ sval = a.w.sval;
  const float4* __restrict__ spp = a.w.spp;
  int by = w.by_lo - 1;
  unsigned i = 0, end = 0, cum = 0;
  unsigned ns = 0, ne = 0;
  row_segment(a, g, w, w.by_lo, ns, ne);
  // moves [i, end) to the next bin row holding part of [lo, hi); false at the end
  auto next_row = [&]() -> bool {
    for (;;) {
      if (++by > w.by_hi || cum >= hi) return false;
      const unsigned s0 = ns, e0 = ne;
      if (by < w.by_hi) row_segment(a, g, w, by + 1, ns, ne);
      const unsigned len = e0 - s0, rs = cum;
      cum += len;
      i = s0 + (lo > rs ? min(lo - rs, len) : 0u);
      end = s0 + (hi > rs ? min(hi - rs, len) : 0u);
      if (i < end && !GMI_IN_BOUNDS(a.w, end - 1u, a.n_total, CK_CAND)) end = i;
      if (i < end) return true;
    }
  };
  if (next_row()) {
    float2 pn = __ldg(&sxy[i]);
    float4 cn = __ldg(&sval[i]);
    float4 sn = PP ? __ldg(&spp[i]) : make_float4(0.f, 0.f, 0.f, 0.f);
    bool more = true;
    while (more) {
      const float2 p = pn;
      const float4 cv = cn;
      const float4 spc = sn;
      if (++i >= end) more = next_row();
      if (more) {
        pn = __ldg(&sxy[i]);
        cn = __ldg(&sval[i]);
        if (PP) sn = __ldg(&spp[i]);
      }
      consume(p, cv, spc);
    }
  }
}

}  // namespace gmi
