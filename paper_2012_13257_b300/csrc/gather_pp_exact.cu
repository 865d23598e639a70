// Exact mode with a sigma (or covariance) per point: Eq. 1 and Eq. 2 with
// point i the normal N(mu_i, S_i), its normaliser kept, over all points.
//
// In log2 units point i weighs lw_i(q) = la_i - Q_i(q), with la_i = log2(
// sigma_b^2 / sqrt(det S_i)) >= 0 (sigma_b the bound given with the call) and
// Q_i = d^T S_i^-1 d log2(e) / 2 (pp_consts, pp_cov_consts).  A pixel's
// weights are evaluated relative to its largest one, L(q) = max_i lw_i(q), so
// that no sum underflows to 0/0 however far the pixel is from the points; den
// is sum_i 2^(lw_i - L(q)) and shift the largest weight's natural log in the
// normalisation of the oracle (ln w_i with w_i = exp(-Q/2) / sqrt(det S_i)).
// A point weighing less than e^{-k^2/2} of the largest may be skipped (the
// rule of shared-sigma exact mode); every point within the radius below is
// summed.
//
// One warp per micro-tile, lanes = (pixel, part) as in the far-field kernel:
//   A. a lower bound Lt on L(q) over the micro-tile: the largest weight of the
//      points of the smallest non-empty bin window, at the tile's pixels;
//   B. candidates: a point can reach lw_i(q) >= Lt - k^2 log2(e) / 2 only
//      within R^2 = (la_max - Lt + k^2 log2(e) / 2) / kappa_b of the tile
//      (Q_i >= kappa_b d^2 since every S_i's largest eigenvalue is at most
//      sigma_b^2, and la_i <= la_max, the image's largest, found by the scatter);
//   C. L(q) = max over the candidates, in FP32 where every quadratic form the
//      tile needs stays small, else in FP64 from the raw sigmas (far from the
//      points lw is large and the differences lw_i - L(q) small);
//   D. sums of 2^(lw_i - L(q)) and of those weights times the colours.
// The backward pass recomputes C and D per pixel and adds every pair's
// gradient terms atomically into per-point moments, turned into gradients by
// a finishing kernel.
#include "api_internal.h"
#include "bwd_args.h"
#include "far_collect.cuh"

namespace gmi {

// lw_i(q) in log2 units at the offset (dx, dy) = q - mu_i from point i's
// constants (pp_consts: PPK 1; pp_cov_consts: PPK 2), in FP32.  Accurate to
// a few 1e-7 of the quadratic form, enough while the forms a micro-tile needs
// stay below kPpNarrowQ.
template <int PPK>
__device__ __forceinline__ float pp_lw_f(const float4 k, float dx, float dy) {
  if (PPK == 2) return k.w - (k.x * dx * dx + k.y * dx * dy + k.z * dy * dy);
  const float u = k.x * dx, v = k.y * dy;
  return k.z - (u * u + v * v);
}

constexpr float kPpNarrowQ = 64.0f;

// lw_i(q) in FP64 from the raw sigmas (point i found through the scatter's
// permutation) and the exact offset: far from the points the forms are large
// and the weights a pixel sums differ by small differences of them, which
// FP32 constants and offsets would blur.  The normaliser la_i stays FP32
// (its error does not grow with the distance).
template <int PPK>
__device__ __forceinline__ double pp_lw_d(const KArgs& a, const ImageGeom& g, unsigned idx, const float4 k,
                                          float qx, float qy, float2 p) {
  constexpr double kHalfLog2e = 0.72134752044448170;   // log2(e) / 2
  const float* sg = g.sigmas + (long long)g.pp_kind * a.w.perm[idx];
  const double x = (double)qx - (double)p.x, y = (double)qy - (double)p.y;
  double q;
  if (g.pp_kind == 3) {
    const double u = x / (double)sg[0], v = y / (double)sg[1], r = sg[2];
    q = (u * u - 2.0 * r * u * v + v * v) / (1.0 - r * r);
  } else {
    const double sx = sg[0], sy = g.pp_kind == 2 ? (double)sg[1] : sx;
    const double u = x / sx, v = y / sy;
    q = u * u + v * v;
  }
  return (double)(PPK == 2 ? k.w : k.z) - q * kHalfLog2e;
}

// The summed-area table of the bin counts (the smallest-window search reads
// it), as a kernel of its own: no near kernel runs in this mode.
__global__ void __launch_bounds__(128) pp_sat_kernel(KArgs a) {
  if (bins_invalid(a.w.status)) return;
  sat_build(a);
}

// Per-micro-tile state of steps A and B: the candidate radius, whether the
// quadratic forms can exceed kPpNarrowQ (then FP64), and whether the image
// holds any point.
struct PpWindow {
  FarTile t;
  float R, R2;
  bool any, wide;
};

template <int PPK>
__device__ PpWindow pp_window(const KArgs& a, const ImageGeom& g, int x0, int y0, int nx, int ny, bool valid, float qx,
                              float qy, int PS, int part, int nparts, unsigned* L) {
  const unsigned full = 0xffffffffu;
  PpWindow w;
  w.t.xa = (float)x0 + 0.5f;
  w.t.xb = (float)(x0 + nx) - 0.5f;
  w.t.ya = (float)y0 + 0.5f;
  w.t.yb = (float)(y0 + ny) - 0.5f;
  w.R = w.R2 = 0.0f;
  w.wide = false;
  const float hi = smallest_window(a, g, w.t);
  w.any = hi >= 0.0f;
  if (!w.any) return w;
  // A. the largest weight of the window's points at this pixel (a lower
  // bound on its L), then the smallest over the tile's pixels
  const unsigned ns = min(collect(a, g, w.t, hi, -1.0f, 0u, L), (unsigned)kFarCap);
  float l0 = -INFINITY;
  for (unsigned k = part; k < ns; k += nparts) {
    const unsigned idx = L[k];
    const float2 p = a.w.sxy[idx];
    l0 = fmaxf(l0, pp_lw_f<PPK>(a.w.spp[idx], qx - p.x, qy - p.y));
  }
  for (int o = PS; o < 32; o <<= 1) l0 = fmaxf(l0, __shfl_xor_sync(full, l0, o));
  float Lt = valid ? l0 : INFINITY;
  for (int o = 16; o > 0; o >>= 1) Lt = fminf(Lt, __shfl_xor_sync(full, Lt, o));
  Lt -= 1e-3f * (1.0f + fabsf(Lt));   // below the float rounding of the bound
  __syncwarp();
  // B. the radius within which a point can come within e^{-k^2/2} of Lt;
  // every quadratic form such a point takes is at most qmax
  const float la_max = __uint_as_float(a.w.status[kLaMax]);
  const float qmax = la_max - Lt + g.e_trunc;
  w.wide = !(qmax <= kPpNarrowQ);
  w.R2 = qmax / g.kappa * (1.0f + 1e-5f) + 1e-5f;
  w.R = sqrtf(w.R2);
  return w;
}

// Steps C and D for the lane's pixel and its share (part) of the candidates:
// Lq = the pixel's largest log2 weight and acc = (den, numerators) of the
// weights 2^(lw_i - Lq), summed over the parts.  L holds the last chunk of the
// candidate list on return.
template <int C, int PPK>
__device__ __forceinline__ void pp_pixel_sums(const KArgs& a, const ImageGeom& g, const PpWindow& w, float qx,
                                              float qy, int PS, int part, int nparts, unsigned total, unsigned* L,
                                              double& Lq, float* acc) {
  const unsigned full = 0xffffffffu;
  Lq = -INFINITY;
  for (unsigned skip = 0; skip < total; skip += kFarCap) {
    if (skip > 0) collect(a, g, w.t, w.R, w.R2, skip, L);
    const unsigned n = min(total - skip, (unsigned)kFarCap);
    if (w.wide) {
      for (unsigned k = part; k < n; k += nparts) {
        const unsigned idx = L[k];
        Lq = fmax(Lq, pp_lw_d<PPK>(a, g, idx, a.w.spp[idx], qx, qy, a.w.sxy[idx]));
      }
    } else {
      float lf = -INFINITY;
      for (unsigned k = part; k < n; k += nparts) {
        const unsigned idx = L[k];
        const float2 p = a.w.sxy[idx];
        lf = fmaxf(lf, pp_lw_f<PPK>(a.w.spp[idx], qx - p.x, qy - p.y));
      }
      Lq = fmax(Lq, (double)lf);
    }
    __syncwarp();
  }
  for (int o = PS; o < 32; o <<= 1) Lq = fmax(Lq, __shfl_xor_sync(full, Lq, o));
  const float Lf = (float)Lq;
#pragma unroll
  for (int k = 0; k <= kMaxC; ++k) acc[k] = 0.0f;
  for (unsigned skip = 0; skip < total; skip += kFarCap) {
    if (skip > 0 || total > (unsigned)kFarCap) collect(a, g, w.t, w.R, w.R2, skip, L);
    const unsigned n = min(total - skip, (unsigned)kFarCap);
    for (unsigned k = part; k < n; k += nparts) {
      const unsigned idx = L[k];
      const float2 p = a.w.sxy[idx];
      const float4 kk = a.w.spp[idx];
      const float e = w.wide ? (float)(pp_lw_d<PPK>(a, g, idx, kk, qx, qy, p) - Lq)
                             : pp_lw_f<PPK>(kk, qx - p.x, qy - p.y) - Lf;
      const float wt = ex2(e);
      const float4 cv = a.w.sval[idx];
      acc[0] += wt;
      acc[1] = fmaf(wt, cv.x, acc[1]);
      if (C > 1) acc[2] = fmaf(wt, cv.y, acc[2]);
      if (C > 2) acc[3] = fmaf(wt, cv.z, acc[3]);
      if (C > 3) acc[4] = fmaf(wt, cv.w, acc[4]);
    }
    __syncwarp();
  }
#pragma unroll
  for (int k = 0; k <= C; ++k)
    for (int o = PS; o < 32; o <<= 1) acc[k] += __shfl_xor_sync(full, acc[k], o);
}

template <int C, int PPK>
__global__ void __launch_bounds__(32 * kFarWarps) pp_exact_kernel(KArgs a, int mth, int mtw) {
  __shared__ unsigned lists[kFarWarps][kFarCap];
  if (bins_invalid(a.w.status)) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned* L = lists[wid];
  const ImageGeom g = a.g0;
  const int PS = mth * mtw, nparts = 32 / PS;
  const int slot = lane % PS, part = lane / PS;
  const int pr = slot / mtw, pj = slot % mtw;
  const long long n_mt = (long long)g.mtx * g.mty;
  const double ln2 = 0.69314718055994531;
  const double shift_off = 2.0 * log((double)g.sigma);   // ln sigma_b^2: to the oracle's normalisation
  for (long long mt = (long long)blockIdx.x * kFarWarps + wid; mt < n_mt; mt += (long long)gridDim.x * kFarWarps) {
    const int x0 = (int)(mt % g.mtx) * mtw, y0 = (int)(mt / g.mtx) * mth;
    const int nx = min(mtw, g.W - x0), ny = min(mth, g.H - y0);
    const bool valid = pr < ny && pj < nx;
    const float qx = (float)(x0 + pj) + 0.5f, qy = (float)(y0 + pr) + 0.5f;
    const PpWindow w = pp_window<PPK>(a, g, x0, y0, nx, ny, valid, qx, qy, PS, part, nparts, L);
    float acc[kMaxC + 1];
#pragma unroll
    for (int k = 0; k <= kMaxC; ++k) acc[k] = 0.0f;
    double Lq = -INFINITY;
    if (w.any) {
      const unsigned total = collect(a, g, w.t, w.R, w.R2, 0u, L);
      pp_pixel_sums<C, PPK>(a, g, w, qx, qy, PS, part, nparts, total, L, Lq, acc);
    }
    if (valid && part == 0) {
      const long long pix = (long long)(y0 + pr) * g.W + (x0 + pj);
      const float inv = acc[0] > 0.0f ? __frcp_rn(acc[0]) : 0.0f;
#pragma unroll
      for (int ch = 0; ch < C; ++ch) g.image[pix * C + ch] = acc[1 + ch] * inv;
      if (g.den) g.den[pix] = acc[0];
      if (g.shift) g.shift[pix] = w.any ? (float)(Lq * ln2 - shift_off) : 0.0f;
    }
    __syncwarp();   // the candidate list is rewritten by the next micro-tile
  }
}

constexpr int kPpMoments = kPpMomentFloats;   // per point: A_0..A_3, Bx, By, Sxx, Sxy, Syy, S

// Backward: per micro-tile, the forward's L(q), den and colour again, then
// every (pixel, candidate) pair adds, with w = 2^(lw_i - L(q)) / den and
// t = sum_c g_c (c_{i,c} - c_c(q)):  A_c += w g_c, and with wt = w t,
// Bx += wt dx, By += wt dy, Sxx += wt dx^2, Sxy += wt dx dy, Syy += wt dy^2,
// S += wt  (d = q - mu_i), summed over the part's pixels by shuffles and added
// to the point's moments by one lane (atomics).
template <int C, int PPK>
__global__ void __launch_bounds__(32 * kFarWarps) pp_exact_bwd_kernel(KArgs a, int mth, int mtw, const float* grad,
                                                                      float* mom) {
  __shared__ unsigned lists[kFarWarps][kFarCap];
  if (bins_invalid(a.w.status)) return;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned* L = lists[wid];
  const ImageGeom g = a.g0;
  const int PS = mth * mtw, nparts = 32 / PS;
  const int slot = lane % PS, part = lane / PS;
  const int pr = slot / mtw, pj = slot % mtw;
  const long long n_mt = (long long)g.mtx * g.mty;
  const unsigned pmask = PS == 32 ? full : ((1u << PS) - 1u) << (part * PS);
  for (long long mt = (long long)blockIdx.x * kFarWarps + wid; mt < n_mt; mt += (long long)gridDim.x * kFarWarps) {
    const int x0 = (int)(mt % g.mtx) * mtw, y0 = (int)(mt / g.mtx) * mth;
    const int nx = min(mtw, g.W - x0), ny = min(mth, g.H - y0);
    const bool valid = pr < ny && pj < nx;
    const float qx = (float)(x0 + pj) + 0.5f, qy = (float)(y0 + pr) + 0.5f;
    const PpWindow w = pp_window<PPK>(a, g, x0, y0, nx, ny, valid, qx, qy, PS, part, nparts, L);
    if (!w.any) continue;
    const unsigned total = collect(a, g, w.t, w.R, w.R2, 0u, L);
    // the pixel's largest log-weight, den and colour, as the forward formed them
    double Lq;
    float acc[kMaxC + 1];
    pp_pixel_sums<C, PPK>(a, g, w, qx, qy, PS, part, nparts, total, L, Lq, acc);
    const float Lf = (float)Lq;
    // G_c = g_c / den and s' = sum_c G_c c_c(q) of this lane's pixel
    float G[4] = {0.f, 0.f, 0.f, 0.f}, sp = 0.0f;
    if (valid && acc[0] > 0.0f) {
      const float inv = __frcp_rn(acc[0]);
      const long long pix = (long long)(y0 + pr) * g.W + (x0 + pj);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        G[c] = grad[pix * C + c] * inv;
        sp = fmaf(G[c], acc[1 + c] * inv, sp);
      }
    }
    if (total > (unsigned)kFarCap) collect(a, g, w.t, w.R, w.R2, 0u, L);
    for (unsigned skip = 0; skip < total; skip += kFarCap) {
      if (skip > 0) collect(a, g, w.t, w.R, w.R2, skip, L);
      const unsigned n = min(total - skip, (unsigned)kFarCap);
      for (unsigned k0 = 0; k0 < n; k0 += nparts) {
        const unsigned k = k0 + part;
        float m[kPpMoments];
#pragma unroll
        for (int j = 0; j < kPpMoments; ++j) m[j] = 0.0f;
        unsigned idx = 0;
        if (k < n) {
          idx = L[k];
          if (valid) {
            const float2 p = a.w.sxy[idx];
            const float4 kk = a.w.spp[idx];
            const float dx = qx - p.x, dy = qy - p.y;
            const float e = w.wide ? (float)(pp_lw_d<PPK>(a, g, idx, kk, qx, qy, p) - Lq)
                                   : pp_lw_f<PPK>(kk, dx, dy) - Lf;
            const float wr = ex2(e);
            const float4 cv = a.w.sval[idx];
            const float c4[4] = {cv.x, cv.y, cv.z, cv.w};
            float tq = -sp;
#pragma unroll
            for (int c = 0; c < C; ++c) {
              tq = fmaf(G[c], c4[c], tq);
              m[c] = wr * G[c];
            }
            const float wt = wr * tq;
            m[4] = wt * dx;
            m[5] = wt * dy;
            m[6] = m[4] * dx;
            m[7] = m[4] * dy;
            m[8] = m[5] * dy;
            m[9] = wt;
          }
        }
#pragma unroll
        for (int j = 0; j < kPpMoments; ++j)
          for (int o = PS >> 1; o > 0; o >>= 1) m[j] += __shfl_xor_sync(full, m[j], o);
        const bool any = (__ballot_sync(full, k < n && valid) & pmask) != 0u;
        if (slot == 0 && any && GMI_IN_BOUNDS(a.w, idx, a.n_total, CK_MOMENT)) {
          float* dst = mom + (size_t)idx * kPpMoments;
#pragma unroll
          for (int j = 0; j < kPpMoments; ++j)
            if (j >= C && j < 4) continue;
            else if (m[j] != 0.0f) atomicAdd(&dst[j], m[j]);
        }
      }
      __syncwarp();
    }
  }
}

// Moments to gradients, one thread per bin-sorted point (written at its input
// index): with e = 1 - rho^2 (rho = 0 for isotropic and axis-aligned sigmas),
//   dL/dmu  = S_i^-1 (Bx, By)
//   dL/dsx  = (Sxx / sx^3 - rho Sxy / (sx^2 sy)) / e - S / sx     (sy likewise)
//   dL/drho = (Sxy / (sx sy) - rho SQ + rho S) / e,
//   SQ = (Sxx / sx^2 - 2 rho Sxy / (sx sy) + Syy / sy^2) / e;
// an isotropic sigma_i gets dL/dsx + dL/dsy.
template <int C>
__global__ void __launch_bounds__(256) pp_exact_finish_kernel(KArgs a, BwdImage bi, const float* mom) {
  if (bins_invalid(a.w.status)) return;
  const ImageGeom g = a.g0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n_total;
       i += (long long)gridDim.x * blockDim.x) {
    const float* m = mom + (size_t)i * kPpMoments;
    const unsigned o = a.w.perm[i];
    const int kind = g.pp_kind;
    const float sx = g.sigmas[(long long)kind * o];
    const float sy = kind >= 2 ? g.sigmas[(long long)kind * o + 1] : sx;
    const float rho = kind == 3 ? g.sigmas[3LL * o + 2] : 0.0f;
    if (bi.gvals) {
#pragma unroll
      for (int c = 0; c < C; ++c) bi.gvals[(long long)o * C + c] = m[c];
    }
    const float Bx = m[4], By = m[5], Sxx = m[6], Sxy = m[7], Syy = m[8], S = m[9];
    const float isx = 1.0f / sx, isy = 1.0f / sy, ie = 1.0f / fmaf(-rho, rho, 1.0f);
    if (bi.gpts) {
      bi.gpts[2LL * o] = (Bx * isx * isx - rho * By * isx * isy) * ie;
      bi.gpts[2LL * o + 1] = (By * isy * isy - rho * Bx * isx * isy) * ie;
    }
    if (bi.gsigs) {
      const float gsx = (Sxx * isx * isx * isx - rho * Sxy * isx * isx * isy) * ie - S * isx;
      const float gsy = (Syy * isy * isy * isy - rho * Sxy * isx * isy * isy) * ie - S * isy;
      if (kind == 1) {
        bi.gsigs[o] = gsx + gsy;
      } else if (kind == 2) {
        bi.gsigs[2LL * o] = gsx;
        bi.gsigs[2LL * o + 1] = gsy;
      } else {
        const float sq = (Sxx * isx * isx - 2.0f * rho * Sxy * isx * isy + Syy * isy * isy) * ie;
        bi.gsigs[3LL * o] = gsx;
        bi.gsigs[3LL * o + 1] = gsy;
        bi.gsigs[3LL * o + 2] = (Sxy * isx * isy - rho * sq + rho * S) * ie;
      }
    }
  }
}

static int sat_grid(const KArgs& a) {
  const long long warps = a.satj_total > 0 ? a.satj_total : 1;
  return (int)std::min<long long>((warps + 3) / 4, (long long)device_sm_count() * 8);
}

// Resident blocks per SM of a kernel (1 if the query fails), computed once
// per instantiation; warm_pp_exact fills them before any stream capture.
template <typename K>
static int blocks_per_sm(K kernel) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, 32 * kFarWarps, 0) != cudaSuccess || n < 1) n = 1;
  return n;
}

template <int C, int PPK>
static int fwd_per_sm() {
  static const int n = blocks_per_sm(pp_exact_kernel<C, PPK>);
  return n;
}

template <int C, int PPK>
static int bwd_per_sm() {
  static const int n = blocks_per_sm(pp_exact_bwd_kernel<C, PPK>);
  return n;
}

// One persistent wave of warps over the micro-tiles, no more than they need.
static int pp_grid(const KArgs& a, int per_sm) {
  const long long need = ((long long)a.g0.mtx * a.g0.mty + kFarWarps - 1) / kFarWarps;
  return (int)std::max<long long>(1, std::min<long long>(need, (long long)device_sm_count() * per_sm));
}

template <int C, int PPK>
static cudaError_t pp_exact_fwd_c(const KArgs& a, int mth, int mtw, cudaStream_t s) {
  pp_sat_kernel<<<sat_grid(a), 128, 0, s>>>(a);
  pp_exact_kernel<C, PPK><<<pp_grid(a, fwd_per_sm<C, PPK>()), 32 * kFarWarps, 0, s>>>(a, mth, mtw);
  return cudaGetLastError();
}

// Exact-mode forward with per-point sigmas on a binned single image (spp and
// the largest normaliser written by the scatter); ppk 1 separable, 2 full.
cudaError_t launch_pp_exact_forward(const KArgs& a, int mth, int mtw, int ppk, cudaStream_t s) {
  switch (a.C * 4 + (ppk == 2 ? 1 : 0)) {
    case 4: return pp_exact_fwd_c<1, 1>(a, mth, mtw, s);
    case 5: return pp_exact_fwd_c<1, 2>(a, mth, mtw, s);
    case 8: return pp_exact_fwd_c<2, 1>(a, mth, mtw, s);
    case 9: return pp_exact_fwd_c<2, 2>(a, mth, mtw, s);
    case 12: return pp_exact_fwd_c<3, 1>(a, mth, mtw, s);
    case 13: return pp_exact_fwd_c<3, 2>(a, mth, mtw, s);
    case 16: return pp_exact_fwd_c<4, 1>(a, mth, mtw, s);
    default: return pp_exact_fwd_c<4, 2>(a, mth, mtw, s);
  }
}

template <int C, int PPK>
static void warm_c() {
  fwd_per_sm<C, PPK>();
  bwd_per_sm<C, PPK>();
}

void warm_pp_exact(int C, int ppk) {
  switch (C * 4 + (ppk == 2 ? 1 : 0)) {
    case 4: warm_c<1, 1>(); break;
    case 5: warm_c<1, 2>(); break;
    case 8: warm_c<2, 1>(); break;
    case 9: warm_c<2, 2>(); break;
    case 12: warm_c<3, 1>(); break;
    case 13: warm_c<3, 2>(); break;
    case 16: warm_c<4, 1>(); break;
    default: warm_c<4, 2>(); break;
  }
}

template <int C, int PPK>
static cudaError_t pp_exact_bwd_c(const KArgs& a, const BwdImage& bi, int mth, int mtw, float* mom, cudaStream_t s) {
  pp_sat_kernel<<<sat_grid(a), 128, 0, s>>>(a);
  if (cudaMemsetAsync(mom, 0, sizeof(float) * kPpMoments * (size_t)a.n_total, s) != cudaSuccess)
    return cudaErrorUnknown;
  pp_exact_bwd_kernel<C, PPK><<<pp_grid(a, bwd_per_sm<C, PPK>()), 32 * kFarWarps, 0, s>>>(a, mth, mtw, bi.grad, mom);
  const unsigned blocks = (unsigned)std::max<long long>(1, std::min<long long>((a.n_total + 255) / 256, 4096));
  pp_exact_finish_kernel<C><<<blocks, 256, 0, s>>>(a, bi, mom);
  return cudaGetLastError();
}

// Exact-mode backward with per-point sigmas: mom holds kPpMoments floats per point.
cudaError_t launch_pp_exact_backward(const KArgs& a, const BwdImage& bi, int mth, int mtw, int ppk, float* mom,
                                     cudaStream_t s) {
  switch (a.C * 4 + (ppk == 2 ? 1 : 0)) {
    case 4: return pp_exact_bwd_c<1, 1>(a, bi, mth, mtw, mom, s);
    case 5: return pp_exact_bwd_c<1, 2>(a, bi, mth, mtw, mom, s);
    case 8: return pp_exact_bwd_c<2, 1>(a, bi, mth, mtw, mom, s);
    case 9: return pp_exact_bwd_c<2, 2>(a, bi, mth, mtw, mom, s);
    case 12: return pp_exact_bwd_c<3, 1>(a, bi, mth, mtw, mom, s);
    case 13: return pp_exact_bwd_c<3, 2>(a, bi, mth, mtw, mom, s);
    case 16: return pp_exact_bwd_c<4, 1>(a, bi, mth, mtw, mom, s);
    default: return pp_exact_bwd_c<4, 2>(a, bi, mth, mtw, mom, s);
  }
}

}  // namespace gmi
