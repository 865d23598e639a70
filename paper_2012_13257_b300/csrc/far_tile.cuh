// One far-field micro-tile (an entry of the far-field queue): exact Eq. 1 /
// Eq. 2 for pixels far from every known point, the weights taken relative to
// each pixel's nearest squared distance.  Shared by the far kernel and the
// staged near kernel's warps once they run out of near work.
//   A. bracket the smallest Chebyshev window around the micro-tile that holds
//      any point (doubling, then bisection, on summed-area-table counts) and
//      bound U >= max_q m_q with up to kFarCap of those points;
//   B. collect every point within Euclidean distance R = sqrt(U + k^2 sigma^2)
//      of the micro-tile (indices in L, in chunks if many);
//   C. per pixel, m~_q = min d^2 over the candidates (float32);
//   D. per pixel, sum w = 2^(-kappa e) c over candidates in the shell, with
//      e = d^2 - m~_q from error-free transformations (common.cuh).
// Lanes are split as (pixel slot, part): pixels of the micro-tile times
// 32 / (mth * mtw) interleaved parts of the candidate list, combined with
// shuffles in a fixed order (the result does not depend on scheduling).
// One warp; L: kFarCap indices of this warp's shared memory.
#pragma once

#include "far_collect.cuh"

namespace gmi {

template <int C>
__device__ __forceinline__ void far_entry(const KArgs& a, int mth, int mtw, const uint2 q, unsigned* L) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int PS = mth * mtw;              // pixel slots: 8, 16 or 32
  const int nparts = 32 / PS;
  const int slot = lane % PS, part = lane / PS;
  const int pr = slot / mtw, pj = slot % mtw;
  const int img = GMI_IN_BOUNDS(a.w, q.x, a.n_images, CK_FARQ_READ) ? (int)q.x : 0;
  const ImageGeom g = a.w.table ? a.w.table[img] : a.g0;
  const int mt_x = (int)(q.y % (unsigned)g.mtx), mt_y = (int)(q.y / (unsigned)g.mtx);
  const int x0 = mt_x * mtw, y0 = mt_y * mth;
  const int nx = min(mtw, g.W - x0), ny = min(mth, g.H - y0);
  FarTile t;
  t.xa = (float)x0 + 0.5f;
  t.xb = (float)(x0 + nx) - 0.5f;
  t.ya = (float)y0 + 0.5f;
  t.yb = (float)(y0 + ny) - 0.5f;
  const bool valid = pr < ny && pj < nx;
  const float qx = (float)(x0 + pj) + 0.5f, qy = (float)(y0 + pr) + 0.5f;

  // A. smallest non-empty window (bin resolution), then U from its points
  const float hi = smallest_window(a, g, t);
  float accd[kMaxC + 1];
#pragma unroll
  for (int k = 0; k <= kMaxC; ++k) accd[k] = 0.0f;
  float mshift = 0.0f;
  if (hi >= 0.0f) {
    const unsigned ns = min(collect(a, g, t, hi, -1.0f, 0u, L), (unsigned)kFarCap);
    float best = INFINITY;
    for (unsigned k = part; k < ns; k += nparts) {
      const float2 p = a.w.sxy[L[k]];
      const float dx = qx - p.x, dy = qy - p.y;
      best = fminf(best, fmaf(dx, dx, dy * dy));
    }
    for (int o = PS; o < 32; o <<= 1) best = fminf(best, __shfl_xor_sync(full, best, o));
    float U = valid ? best : 0.0f;
    for (int o = 16; o > 0; o >>= 1) U = fmaxf(U, __shfl_xor_sync(full, U, o));
    __syncwarp();

    // B. candidates within R of the micro-tile
    const float R2 = (U + g.r2k) * (1.0f + 1e-6f) + 1e-6f;
    const float R = sqrtf(R2);
    const unsigned total = collect(a, g, t, R, R2, 0u, L);

    // C. nearest squared distance per pixel
    float m = INFINITY;
    for (unsigned skip = 0; skip < total; skip += kFarCap) {
      if (skip > 0) collect(a, g, t, R, R2, skip, L);
      const unsigned n = min(total - skip, (unsigned)kFarCap);
      for (unsigned k = part; k < n; k += nparts) {
        const float2 p = a.w.sxy[L[k]];
        const float dx = qx - p.x, dy = qy - p.y;
        m = fminf(m, fmaf(dx, dx, dy * dy));
      }
      __syncwarp();
    }
    for (int o = PS; o < 32; o <<= 1) m = fminf(m, __shfl_xor_sync(full, m, o));
    mshift = m;

    // D. shell sum with shifted, compensated exponents
    const float thr = (m + g.r2k) * (1.0f + 4e-7f) + 1e-30f;
    for (unsigned skip = 0; skip < total; skip += kFarCap) {
      if (skip > 0 || total > (unsigned)kFarCap) collect(a, g, t, R, R2, skip, L);
      const unsigned n = min(total - skip, (unsigned)kFarCap);
      for (unsigned k = part; k < n; k += nparts) {
        const unsigned idx = L[k];
        const float2 p = a.w.sxy[idx];
        const float dx = qx - p.x, dy = qy - p.y;
        if (fmaf(dx, dx, dy * dy) <= thr) {
          const float ee = shifted_sqdist(qx, qy, p.x, p.y, m);
          const float w = ex2(-g.kappa * ee);
          const float4 cv = a.w.sval[idx];
          accd[0] += w;
          accd[1] = fmaf(w, cv.x, accd[1]);
          if (C > 1) accd[2] = fmaf(w, cv.y, accd[2]);
          if (C > 2) accd[3] = fmaf(w, cv.z, accd[3]);
          if (C > 3) accd[4] = fmaf(w, cv.w, accd[4]);
        }
      }
      __syncwarp();
    }
#pragma unroll
    for (int k = 0; k <= C; ++k)
      for (int o = PS; o < 32; o <<= 1) accd[k] += __shfl_xor_sync(full, accd[k], o);
  }
  if (valid && part == 0) {
    const long long pix = (long long)(y0 + pr) * g.W + (x0 + pj);
    const float inv = accd[0] > 0.0f ? 1.0f / accd[0] : 0.0f;
#pragma unroll
    for (int ch = 0; ch < C; ++ch) g.image[pix * C + ch] = accd[1 + ch] * inv;
    if (g.den) g.den[pix] = accd[0];
    if (g.shift) g.shift[pix] = mshift;
  }
}

}  // namespace gmi
