// Candidate collection around a micro-tile, shared by the far-field forward
// kernel and the backward fallback kernel: Chebyshev windows over the bin
// grid, counted (summed-area table) or enumerated one warp at a time.
#pragma once

#include "sat.cuh"

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

// Half-width (a multiple of the bin edge) of the smallest Chebyshev window
// around t, at bin resolution, that holds any point; -1 when the image has
// none.  Every count comes from the summed-area table (four loads), one
// window per lane: a pass of doubling half-widths b 2^lane, then bisection
// passes of 32 evenly spaced half-widths between the largest empty and the
// smallest non-empty window found so far.
static __device__ float smallest_window(const KArgs& a, const ImageGeom& g, const FarTile& t) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const float bf = (float)g.b;
  auto nonempty = [&](float h) {
    int bx_lo, bx_hi, by_lo, by_hi;
    window_bins(g, t, h, bx_lo, bx_hi, by_lo, by_hi);
    return sat_count(a, g, bx_lo, bx_hi, by_lo, by_hi) > 0u;
  };
  const unsigned nz = __ballot_sync(full, nonempty(ldexpf(bf, lane)));
  if (nz == 0u) return -1.0f;
  const int k = __ffs(nz) - 1;
  float hi = ldexpf(bf, k);
  float lo = k > 0 ? ldexpf(bf, k - 1) : 0.0f;   // window lo is empty (or lo == 0), window hi is not
  while (hi - lo > bf) {
    const float step = fmaxf(bf, floorf((hi - lo) / (32.0f * bf)) * bf);
    const unsigned m = __ballot_sync(full, nonempty(fminf(lo + (float)(lane + 1) * step, hi)));
    const int j = m ? __ffs(m) - 1 : 32;
    const float nlo = j > 0 ? fminf(lo + (float)j * step, hi) : lo;
    const float nhi = j < 32 ? fminf(lo + (float)(j + 1) * step, hi) : hi;
    if (nhi - nlo >= hi - lo) break;   // no progress (cannot happen; guards the loop)
    lo = nlo;
    hi = nhi;
  }
  return hi;
}

// Appends to L the indices of the points of the Chebyshev window of
// half-width h around t (r2 < 0), or of the points whose squared Euclidean
// distance to the pixel rectangle is at most r2 (then h = sqrt(r2)),
// numbered [skip, skip + kFarCap) in enumeration order (bin rows in order,
// sorted order within a row).  Returns how many points qualify in total.
// For the disc, each bin row's x-range is narrowed by the row's distance to
// the rectangle (border rows, which can hold clamped out-of-frame points, are
// kept whole), and the rows' points are walked as one flat range, 32 per
// step, so that the loads of many rows are in flight together.
static __device__ unsigned collect(const KArgs& a, const ImageGeom& g, const FarTile& t, float h, float r2,
                                   unsigned skip, unsigned* L) {
  int bx_lo, bx_hi, by_lo, by_hi;
  window_bins(g, t, h, bx_lo, bx_hi, by_lo, by_hi);
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  const float bf = (float)g.b;
  unsigned total = 0;
  for (int by0 = by_lo; by0 <= by_hi; by0 += 32) {
    const int myrow = by0 + lane;
    unsigned s = 0, e = 0;
    if (myrow <= by_hi) {
      int xl = bx_lo, xh = bx_hi;
      if (r2 >= 0.0f) {
        float dyr = 0.0f;
        if (myrow > 0 && myrow < g.nby - 1)
          dyr = fmaxf(fmaxf((float)myrow * bf - t.yb, t.ya - (float)(myrow + 1) * bf), 0.0f);
        const float hx = sqrtf(fmaxf(r2 - dyr * dyr, 0.0f));
        xl = bin_coord(t.xa - hx, g.inv_b, g.nbx);
        xh = bin_coord(t.xb + hx, g.inv_b, g.nbx);
      }
      const long long rowb = g.bin_base + (long long)myrow * g.nbx;
      s = a.w.off[rowb + xl];
      e = a.w.off[rowb + xh + 1];
    }
    if (r2 < 0.0f) {
      // the whole window qualifies: positions follow from the row lengths
      const unsigned len = e - s;
      unsigned incl = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += y;
      }
      const unsigned base = total + incl - len;
      for (unsigned k = 0; k < len; ++k) {
        const unsigned pos = base + k;
        if (pos >= skip && pos < skip + kFarCap)
          L[pos - skip] = GMI_IN_BOUNDS(a.w, s + k, a.n_total, CK_CAND) ? s + k : 0u;
      }
      total += __shfl_sync(full, incl, 31);
      continue;
    }
    // the rows' points as one flat range [0, n): prefix of row lengths
    const unsigned len = e - s;
    unsigned incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(full, incl, o);
      if (lane >= o) incl += y;
    }
    const unsigned n = __shfl_sync(full, incl, 31);
    const unsigned excl = incl - len;
    for (unsigned f0 = 0; f0 < n; f0 += 32) {
      const unsigned f = f0 + lane;
      // the row holding flat index f: the last lane whose prefix is <= f
      int r = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const unsigned ex = __shfl_sync(full, excl, r + step);
        if (r + step < 32 && ex <= f) r += step;
      }
      const unsigned rs = __shfl_sync(full, s, r), rex = __shfl_sync(full, excl, r);
      bool pass = false;
      unsigned idx = 0;
      if (f < n && GMI_IN_BOUNDS(a.w, rs + (f - rex), a.n_total, CK_CAND)) {
        idx = rs + (f - rex);
        const float2 p = a.w.sxy[idx];
        const float dx = fmaxf(fmaxf(t.xa - p.x, p.x - t.xb), 0.0f);
        const float dy = fmaxf(fmaxf(t.ya - p.y, p.y - t.yb), 0.0f);
        pass = dx * dx + dy * dy <= r2;
      }
      const unsigned m = __ballot_sync(full, pass);
      const unsigned pos = total + __popc(m & ((1u << lane) - 1u));
      if (pass && pos >= skip && pos < skip + kFarCap) L[pos - skip] = idx;
      total += __popc(m);
    }
  }
  __syncwarp();
  return total;
}

}  // namespace gmi
