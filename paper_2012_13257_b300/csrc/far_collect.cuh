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

// Counts of points in the bins covering K nested Chebyshev windows of
// half-widths h[0] <= ... <= h[K-1], in one pass over the rows of the
// largest (each lane takes rows; the loads of all windows are independent).
template <int K>
static __device__ void window_counts(const KArgs& a, const ImageGeom& g, const FarTile& t, const float (&h)[K],
                                     unsigned (&cnt)[K]) {
  int bx_lo[K], bx_hi[K], by_lo[K], by_hi[K];
#pragma unroll
  for (int k = 0; k < K; ++k) window_bins(g, t, h[k], bx_lo[k], bx_hi[k], by_lo[k], by_hi[k]);
  const int lane = threadIdx.x & 31;
  unsigned s[K];
#pragma unroll
  for (int k = 0; k < K; ++k) s[k] = 0;
  for (int by = by_lo[K - 1] + lane; by <= by_hi[K - 1]; by += 32) {
    const long long rowb = g.bin_base + (long long)by * g.nbx;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (by >= by_lo[k] && by <= by_hi[k]) s[k] += a.w.off[rowb + bx_hi[k] + 1] - a.w.off[rowb + bx_lo[k]];
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    cnt[k] = s[k];
  }
}

// Half-width (a multiple of the bin edge) of the smallest Chebyshev window
// around t, at bin resolution, that holds any point; -1 when none up to hmax.
// Doubling four levels per pass, then eight bisection points per pass.
static __device__ float smallest_window(const KArgs& a, const ImageGeom& g, const FarTile& t) {
  const float bf = (float)g.b;
  const float hmax = 2.0f * (float)max(g.W, g.H) + bf;
  float lo = 0.0f, hi = -1.0f;   // window lo is empty (or lo == 0), window hi is not
  for (float h0 = bf; h0 < 2.0f * hmax; h0 *= 16.0f) {
    const float h[4] = {h0, 2.0f * h0, 4.0f * h0, 8.0f * h0};
    unsigned c[4];
    window_counts<4>(a, g, t, h, c);
    int k = 0;
    while (k < 4 && c[k] == 0) ++k;
    if (k < 4) {
      hi = h[k];
      lo = k > 0 ? h[k - 1] : (h0 > bf ? 0.5f * h0 : 0.0f);
      break;
    }
  }
  if (hi < 0.0f) return -1.0f;
  // bisection at bin resolution: eight evenly spaced half-widths in (lo, hi)
  while (hi - lo > bf) {
    const float step = fmaxf(bf, floorf((hi - lo) / (9.0f * bf)) * bf);
    float h[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) h[j] = fminf(lo + (float)(j + 1) * step, hi);
    unsigned c[8];
    window_counts<8>(a, g, t, h, c);
    int j = 0;
    while (j < 8 && c[j] == 0) ++j;
    const float nlo = j > 0 ? h[j - 1] : lo;
    const float nhi = j < 8 ? h[j] : hi;
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
        if (pos >= skip && pos < skip + kFarCap) L[pos - skip] = s + k;
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
      if (f < n) {
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
