// Backward pass: gradients of L = sum_q sum_c g_c(q) c_c(q) with respect to
// the point colours, the point positions and sigma.  The paper has a backward
// CUDA kernel but prints no formulas; with w_i(q) the weight of point i at
// pixel q, Z_q their sum and t_i(q) = sum_c g_c(q) (c_{i,c} - c_c(q)), the
// chain rule on Eq. 1 gives
//   dL/dc_{i,c} = sum_q g_c(q) w_i(q) / Z_q
//   dL/dmu_i    = sum_q (w_i(q) / Z_q) t_i(q) (q - mu_i) / sigma^2
//   dL/dsigma   = sum_q sum_i (w_i(q) / Z_q) t_i(q) |q - mu_i|^2 / sigma^3.
// From the forward pass only the image c(q), den_q and shift_q are kept
// (w_i(q) / Z_q = 2^(-kappa (d^2 - shift_q)) / den_q); the bins are rebuilt.
//
// With a sigma per point (truncated mode), w_i(q) = 2^(la_i - kx_i dx^2 -
// ky_i dy^2) (pp_consts) and each point has its own terms
//   dL/dx_i  = sum_q (w_i(q) / Z_q) t_i(q) dx / sx_i^2      (y likewise)
//   dL/dsx_i = sum_q (w_i(q) / Z_q) t_i(q) (dx^2 / sx_i^3 - 1 / sx_i),
// the -1/sx_i from the normaliser 1/(sx_i sy_i) of the 2D normal (it no
// longer cancels); an isotropic sigma_i gets the sum of its two axis terms.
// Every pair lies inside its point's ellipse, so the point-centric kernel
// covers all of them.
//
// Work is split by pixel:
//   * core pixels (no shift, den_q >= 2^-12): point-centric.  One thread per
//     bin-sorted point sweeps the disc of pixels within R_core, with
//     kappa R_core^2 = 20 + 12, which holds every pair whose weight is at least
//     2^-20 of its pixel's density sum; the thread owns its point's gradient,
//     so it is stored without atomics.
//     What the cut drops: a point's pairs outside its disc carry together a
//     normalised weight of at most 2 pi sigma^2 2^(-kappa R_core^2) / den_q
//     (the Gaussian tail), i.e. 2 pi sigma^2 2^-20 (6e-6 at sigma = 1) times
//     max |g| for the colour gradient even if every such pixel had the least
//     core density 2^-12; the position and sigma terms carry the extra
//     factors d / sigma^2 and d^2 / sigma^3 of the tail pairs.  Both stay far
//     below the 1e-3 gradient tolerance.
//   * other pixels (sparse neighbourhoods and the far field): one warp per
//     micro-tile holding such pixels collects the points within the largest
//     radius its pixels need, and adds the pairs' contributions atomically
//     (few pairs: these regions are sparse).
#include <string.h>

#include "api_internal.h"
#include "far_collect.cuh"
#include "bwd_args.h"

namespace gmi {

constexpr float kCoreLog2 = 12.0f;   // core pixel: den >= 2^-kCoreLog2 and no shift
constexpr float kRelLog2 = 20.0f;    // pairs below 2^-kRelLog2 of their pixel's den are dropped

__device__ __forceinline__ BwdImage bwd_image(const BwdArgs& b, int img) { return b.table ? b.table[img] : b.one; }

// Per pixel: G_c = g_c / den and s' = sum_c G_c c_c(q) for core pixels (zero
// elsewhere); micro-tiles with a non-core pixel are queued for the fallback.
template <int C>
__global__ void __launch_bounds__(256) bwd_prep_kernel(KArgs a_in, BwdArgs b) {
  const KArgs a = resolve(a_in);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long gp = (long long)blockIdx.x * blockDim.x + threadIdx.x; gp < a.px_total; gp += stride) {
    const int img = find_image<3>(a, gp);
    const ImageGeom g = a.w.table ? a.w.table[img] : a.g0;   // a copy: no address of a local struct
    const BwdImage bi = bwd_image(b, img);
    const long long px = gp - g.px_base;
    if (px == 0 && bi.gsig) *bi.gsig = 0.0f;   // accumulated by the later kernels
    const float d = bi.den[px];
    const float sh = bi.shift ? bi.shift[px] : 0.0f;
    float G[4] = {0.f, 0.f, 0.f, 0.f};
    float sp = 0.0f;
    if (d > 0.0f) {
      const float inv = 1.0f / d;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        G[c] = bi.grad[px * C + c] * inv;
        sp = fmaf(G[c], bi.image[px * C + c], sp);
      }
    }
    const bool core = d > 0.0f && (b.trunc || (sh == 0.0f && d >= exp2f(-kCoreLog2)));
    float4 v0, v1 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!core) {
      v0 = make_float4(0.f, 0.f, 0.f, 0.f);
    } else if (C == 4) {
      v0 = make_float4(G[0], G[1], G[2], G[3]);
      v1.x = sp;
    } else {
      v0 = make_float4(G[0], G[1], G[2], 0.0f);
      if (C == 1) v0.y = 0.0f;
      v0.w = sp;
    }
    a.w.pplane[gp] = v0;
    if (C == 4) a.w.pplane[a.px_total + gp] = v1;
    if (!core && d > 0.0f) {
      const int y = (int)(px / g.W), x = (int)(px % g.W);
      const unsigned mt = (unsigned)((y / a.mth) * g.mtx + x / a.mtw);
      if (atomicOr(&a.w.fbflag[g.mt_base + mt], 1u) == 0u) {
        const unsigned q = atomicAdd(&a.w.status[kFbCount], 1u);
        if (GMI_IN_BOUNDS(a.w, q, a.mt_total, CK_FBQ)) a.w.fbq[q] = make_uint2((unsigned)img, mt);
      }
    }
  }
}

// Single-image sigma gradient: block sum of D -> one partial per block; the
// last block to finish adds the partials in block order.
__device__ void sigma_block_total(const KArgs& a, const BwdArgs& b, float D) {
  const unsigned full = 0xffffffffu;
  __shared__ float red[8];
  __shared__ bool last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) D += __shfl_xor_sync(full, D, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = D;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    a.w.sig_part[blockIdx.x] = t;
    __threadfence();
    last = atomicAdd(&a.w.status[kSigDone], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    float t = 0.0f;
    for (unsigned k = 0; k < gridDim.x; ++k) t += __ldcg(&a.w.sig_part[k]);
    if (b.one.gsig) *b.one.gsig += t * b.one.inv_s3;
  }
}

// Point-centric gradients over core pixels; one thread per bin-sorted point.
template <int C, bool TRUNC, bool PP>
__global__ void __launch_bounds__(256) bwd_point_kernel(KArgs a_in, BwdArgs b, float rcore_log2) {
  static_assert(TRUNC || !PP, "per-point sigma is built for truncated mode only");
  const KArgs a = resolve(a_in);
  if (bins_invalid(a.w.status)) return;
  const unsigned full = 0xffffffffu;
  float D = 0.0f;
  for (long long i0 = (long long)blockIdx.x * blockDim.x; i0 < a.n_total; i0 += (long long)gridDim.x * blockDim.x) {
    const long long i = i0 + threadIdx.x;
    const bool valid = i < a.n_total;
    int img = 0;
    float Dp = 0.0f;
    if (valid) {
      img = find_image<2>(a, i);
      const ImageGeom g = a.w.table ? a.w.table[img] : a.g0;   // a copy: no address of a local struct
      const BwdImage bi = bwd_image(b, img);
      const float4* __restrict__ plane = a.w.pplane + g.px_base;
      const float4* __restrict__ plane2 = a.w.pplane + a.px_total + g.px_base;
      // per-point sigma: (sqrt(kx_i), sqrt(ky_i), la_i) of this point and its own
      // ellipse kx_i dx^2 + ky_i dy^2 <= e_trunc, walked a little wider (the
      // forward's test below decides membership)
      const float4 spc = PP ? a.w.spp[i] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float kx = spc.x * spc.x, ky = spc.y * spc.y;
      const float e_walk = 1.0001f * g.e_trunc;
      const float rcore2 = TRUNC ? g.r2k : rcore_log2 / g.kappa;
      const float neg_thr = -g.e_trunc;
      const float2 p = a.w.sxy[i];
      const float4 cv = a.w.sval[i];
      const float c4[4] = {cv.x, cv.y, cv.z, cv.w};
      float A[4] = {0.f, 0.f, 0.f, 0.f};
      float Bx = 0.0f, By = 0.0f, Sw = 0.0f, Dy = 0.0f;
      const float R = PP ? sqrtf(e_walk / ky) : sqrtf(rcore2);
      const int iy0 = max(0, (int)ceilf(p.y - R - 0.5f));
      const int iy1 = min(g.H - 1, (int)floorf(p.y + R - 0.5f));
      for (int iy = iy0; iy <= iy1; ++iy) {
        const float dy = (float)iy + 0.5f - p.y;
        const float dy2 = dy * dy;
        const float rem = PP ? e_walk - ky * dy2 : rcore2 - dy2;
        if (rem < 0.0f) continue;
        const float h = PP ? sqrtf(rem / kx) : sqrtf(rem);
        const int ix0 = max(0, (int)ceilf(p.x - h - 0.5f));
        const int ix1 = min(g.W - 1, (int)floorf(p.x + h - 0.5f));
        const float4* __restrict__ P = plane + (long long)iy * g.W;
        // per-point sigma: the row factor exactly as the forward kernel forms it
        // from its micro-tile's first pixel centre, so that both keep the same pairs
        float ayp = 0.0f, gyp = 0.0f;
        if (PP) {
          const int y0 = iy & ~(a.mth - 1);
          const float v = ((float)y0 + 0.5f - p.y) * spc.y;
          const float tv = __fmaf_rn((float)(iy - y0), spc.y, v);
          ayp = __fmul_rn(-tv, tv);
          gyp = ex2(__fadd_rn(ayp, spc.z));
        }
        float rowWt = 0.0f;
        float dx = (float)ix0 + 0.5f - p.x;
#pragma unroll 4
        for (int ix = ix0; ix <= ix1; ++ix, dx += 1.0f) {
          const float d2 = fmaf(dx, dx, dy2);
          float w;
          if (PP) {
            const int x0 = ix & ~(a.mtw - 1);
            const float u = ((float)x0 + 0.5f - p.x) * spc.x;
            const float tu = __fmaf_rn((float)(ix - x0), spc.x, u);
            const float ax = __fmul_rn(-tu, tu);
            w = __fadd_rn(ax, ayp) >= neg_thr ? ex2(ax) * gyp : 0.0f;
          } else {
            w = ex2(-g.kappa * d2);
            if (TRUNC && !(d2 <= g.r2k)) w = 0.0f;
          }
          const float4 pv = __ldg(&P[ix]);
          const float Gv[4] = {pv.x, pv.y, pv.z, pv.w};
          const float sp = C == 4 ? __ldg(&plane2[(long long)iy * g.W + ix]).x : pv.w;
          float t = -sp;
#pragma unroll
          for (int c = 0; c < C; ++c) t = fmaf(Gv[c], c4[c], t);
#pragma unroll
          for (int c = 0; c < C; ++c) A[c] = fmaf(w, Gv[c], A[c]);
          const float wt = w * t;
          Bx = fmaf(wt, dx, Bx);
          rowWt += wt;
          Dp = fmaf(wt, PP ? dx * dx : d2, Dp);   // per-point sigma: the x part only
        }
        By = fmaf(rowWt, dy, By);
        if (PP) {
          Sw += rowWt;
          Dy = fmaf(rowWt, dy2, Dy);
        }
      }
      const unsigned o = a.w.perm[i];
      if (PP) {
        // d ln w / d sx = dx^2 / sx^3 - 1 / sx (likewise y); isotropic: their sum
        const float sx = g.sigmas[(long long)g.pp_kind * o];
        const float sy = g.pp_kind == 2 ? g.sigmas[2LL * o + 1] : sx;
        const float isx2 = 1.0f / (sx * sx), isy2 = 1.0f / (sy * sy);
        if (bi.gpts) {
          bi.gpts[2LL * o] = Bx * isx2;
          bi.gpts[2LL * o + 1] = By * isy2;
        }
        if (bi.gsigs) {
          const float gx = (Dp * isx2 - Sw) / sx, gy = (Dy * isy2 - Sw) / sy;
          if (g.pp_kind == 2) {
            bi.gsigs[2LL * o] = gx;
            bi.gsigs[2LL * o + 1] = gy;
          } else {
            bi.gsigs[o] = gx + gy;
          }
        }
      }
      if (bi.gvals) {
#pragma unroll
        for (int c = 0; c < C; ++c) bi.gvals[(long long)o * C + c] = A[c];
      }
      if (bi.gpts && !PP) {
        bi.gpts[2LL * o] = Bx * bi.inv_s2;
        bi.gpts[2LL * o + 1] = By * bi.inv_s2;
      }
    }
    if (PP) continue;   // no shared sigma to reduce into
    if (b.table) {
      // batched: one float atomic per (warp, image) into that image's sigma gradient
      const unsigned same = __match_any_sync(full, valid ? img : -1);
      if (valid) {
        float s2 = 0.0f;
        for (unsigned m = same; m; m &= m - 1) s2 += __shfl_sync(same, Dp, __ffs(m) - 1);
        if ((int)(threadIdx.x & 31) == __ffs(same) - 1) {
          const BwdImage bi = bwd_image(b, img);
          if (bi.gsig) atomicAdd(bi.gsig, s2 * bi.inv_s3);
        }
      }
    } else {
      D += Dp;
    }
  }
  if constexpr (!PP) {
    if (!b.table) sigma_block_total(a, b, D);
  }
}

// Full covariance per point (truncated mode): one thread per bin-sorted point
// walks the bounding rows of its ellipse d^T S_i^-1 d <= k^2 (a little wider)
// and keeps exactly the pairs the forward kept, by the forward's roundings
// from each micro-tile's first pixel centre.  With the moments
// Bx = sum wt dx, By = sum wt dy, Sxx = sum wt dx^2, Sxy = sum wt dx dy,
// Syy = sum wt dy^2, S = sum wt (wt = (w_i / Z_q) t_i(q)) and e = 1 - rho^2:
//   dL/dmu   = S_i^-1 (Bx, By)
//   dL/dsx   = (Sxx / sx^3 - rho Sxy / (sx^2 sy)) / e - S / sx     (sy likewise)
//   dL/drho  = (Sxy / (sx sy) - rho SQ + rho S) / e,
//   SQ = sum wt Q = (Sxx / sx^2 - 2 rho Sxy / (sx sy) + Syy / sy^2) / e.
template <int C>
__global__ void __launch_bounds__(256) bwd_cov_kernel(KArgs a, BwdArgs b) {
  if (bins_invalid(a.w.status)) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n_total;
       i += (long long)gridDim.x * blockDim.x) {
    const ImageGeom& g = a.g0;
    const BwdImage bi = b.one;
    const float4* __restrict__ plane = a.w.pplane;
    const float4* __restrict__ plane2 = a.w.pplane + a.px_total;
    const unsigned o = a.w.perm[i];
    const float sx = g.sigmas[3LL * o], sy = g.sigmas[3LL * o + 1], rho = g.sigmas[3LL * o + 2];
    const float4 kc = a.w.spp[i];   // (kxx, kxy, kyy, la)
    const float neg_thr = -g.e_trunc;
    const float kw = 1.0001f * sqrtf(g.r2k) / g.sigma;   // k, widened
    const float e1 = fmaf(-rho, rho, 1.0f);
    const float2 p = a.w.sxy[i];
    const float4 cv = a.w.sval[i];
    const float c4[4] = {cv.x, cv.y, cv.z, cv.w};
    float A[4] = {0.f, 0.f, 0.f, 0.f};
    float Bx = 0.f, By = 0.f, Sxx = 0.f, Sxy = 0.f, Syy = 0.f, S = 0.f;
    const float ry = kw * sy;
    const int iy0 = max(0, (int)ceilf(p.y - ry - 0.5f));
    const int iy1 = min(g.H - 1, (int)floorf(p.y + ry - 0.5f));
    for (int iy = iy0; iy <= iy1; ++iy) {
      const int y0 = iy & ~(a.mth - 1);
      const float dy = __fadd_rn((float)y0 + 0.5f - p.y, (float)(iy - y0));
      const float ay = __fmul_rn(-__fmul_rn(kc.z, dy), dy);
      const float by = __fmul_rn(-kc.y, dy);
      // the row's chord: |dx/sx - rho dy/sy| <= sqrt(e (k^2 - dy^2/sy^2))
      const float t = dy / sy;
      const float rem = e1 * fmaf(kw, kw, -t * t);
      if (rem < 0.0f) continue;
      const float cx = p.x + rho * sx * t, hw = sx * sqrtf(rem);
      const int ix0 = max(0, (int)ceilf(cx - hw - 0.5f));
      const int ix1 = min(g.W - 1, (int)floorf(cx + hw - 0.5f));
      const float4* __restrict__ P = plane + (long long)iy * g.W;
      float rowWt = 0.f, rowBx = 0.f;
      for (int ix = ix0; ix <= ix1; ++ix) {
        const int x0 = ix & ~(a.mtw - 1);
        const float dx = __fadd_rn((float)x0 + 0.5f - p.x, (float)(ix - x0));
        const float ax = __fmul_rn(-__fmul_rn(kc.x, dx), dx);
        const float e = __fmaf_rn(by, dx, __fadd_rn(ax, ay));
        if (!(e >= neg_thr)) continue;
        const float w = ex2(__fadd_rn(e, kc.w));
        const float4 pv = __ldg(&P[ix]);
        const float Gv[4] = {pv.x, pv.y, pv.z, pv.w};
        const float sp = C == 4 ? __ldg(&plane2[(long long)iy * g.W + ix]).x : pv.w;
        float tq = -sp;
#pragma unroll
        for (int c = 0; c < C; ++c) tq = fmaf(Gv[c], c4[c], tq);
#pragma unroll
        for (int c = 0; c < C; ++c) A[c] = fmaf(w, Gv[c], A[c]);
        const float wt = w * tq;
        rowWt += wt;
        rowBx = fmaf(wt, dx, rowBx);
        Sxx = fmaf(wt * dx, dx, Sxx);
      }
      S += rowWt;
      Bx += rowBx;
      By = fmaf(rowWt, dy, By);
      Sxy = fmaf(rowBx, dy, Sxy);
      Syy = fmaf(rowWt * dy, dy, Syy);
    }
    if (bi.gvals) {
#pragma unroll
      for (int c = 0; c < C; ++c) bi.gvals[(long long)o * C + c] = A[c];
    }
    const float isx = 1.0f / sx, isy = 1.0f / sy, ie = 1.0f / e1;
    if (bi.gpts) {
      bi.gpts[2LL * o] = (Bx * isx * isx - rho * By * isx * isy) * ie;
      bi.gpts[2LL * o + 1] = (By * isy * isy - rho * Bx * isx * isy) * ie;
    }
    if (bi.gsigs) {
      const float sq = (Sxx * isx * isx - 2.0f * rho * Sxy * isx * isy + Syy * isy * isy) * ie;
      bi.gsigs[3LL * o] = (Sxx * isx * isx * isx - rho * Sxy * isx * isx * isy) * ie - S * isx;
      bi.gsigs[3LL * o + 1] = (Syy * isy * isy * isy - rho * Sxy * isx * isy * isy) * ie - S * isy;
      bi.gsigs[3LL * o + 2] = (Sxy * isx * isy - rho * sq + rho * S) * ie;
    }
  }
}

// Non-core pixels: one warp per queued micro-tile.  Its pixels (lanes
// 0 .. PS - 1) put what their pairs need into shared memory; the candidates
// are then taken 32 at a time, one per lane, and each lane walks the
// micro-tile's non-core pixels (the same for every lane, read as shared-memory
// broadcasts), summing its candidate's terms in registers; it then adds them
// to the point's gradients with its own atomics (no cross-lane sums).
template <int C>
__global__ void __launch_bounds__(32 * kFarWarps) bwd_fallback_kernel(KArgs a_in, BwdArgs b) {
  const KArgs a = resolve(a_in);
  if (bins_invalid(a.w.status)) return;
  __shared__ unsigned lists[kFarWarps][kFarCap];
  __shared__ float4 pxG[kFarWarps][32];   // per pixel: G_c = g_c / den
  __shared__ float4 pxQ[kFarWarps][32];   // per pixel: centre x, y, s', pair limit emax
  __shared__ float2 pxS[kFarWarps][32];   // per pixel: shift, sigma-term offset s0
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned* L = lists[wid];
  const unsigned nq = a.w.status[kFbCount];
  const int PS = a.mth * a.mtw;
  const int pr = lane / a.mtw, pj = lane % a.mtw;
  for (;;) {
    unsigned e = 0;
    if (lane == 0) e = atomicAdd(&a.w.status[kFbHead], 1u);
    e = __shfl_sync(full, e, 0);
    if (e >= nq) break;
    const uint2 qe = a.w.fbq[e];
    const int img = GMI_IN_BOUNDS(a.w, qe.x, a.n_images, CK_FBQ) ? (int)qe.x : 0;
    const unsigned mt = qe.y;
    const ImageGeom g = a.w.table ? a.w.table[img] : a.g0;
    const BwdImage bi = bwd_image(b, img);
    const int mt_x = (int)(mt % (unsigned)g.mtx), mt_y = (int)(mt / (unsigned)g.mtx);
    const int x0 = mt_x * a.mtw, y0 = mt_y * a.mth;
    const int nx = min(a.mtw, g.W - x0), ny = min(a.mth, g.H - y0);
    FarTile t;
    t.xa = (float)x0 + 0.5f;
    t.xb = (float)(x0 + nx) - 0.5f;
    t.ya = (float)y0 + 0.5f;
    t.yb = (float)(y0 + ny) - 0.5f;
    const bool valid = lane < PS && pr < ny && pj < nx;
    const float qx = (float)(x0 + pj) + 0.5f, qy = (float)(y0 + pr) + 0.5f;
    const long long px = (long long)(y0 + pr) * g.W + (x0 + pj);
    float d = 0.0f, sh = 0.0f, G[4] = {0.f, 0.f, 0.f, 0.f}, sp = 0.0f;
    bool mine = false;
    if (valid) {
      d = bi.den[px];
      sh = bi.shift[px];
      mine = d > 0.0f && !(sh == 0.0f && d >= exp2f(-kCoreLog2));
      if (mine) {
        const float inv = 1.0f / d;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          G[c] = bi.grad[px * C + c] * inv;
          sp = fmaf(G[c], bi.image[px * C + c], sp);
        }
      }
    }
    // this pixel keeps pairs with kappa (d^2 - shift) <= kRelLog2 - log2(den)
    const float emax = mine ? (kRelLog2 - log2f(d)) / g.kappa : 0.0f;
    // sum_i (w_i / Z) t_i = 0 at every pixel, so the sigma term may use
    // d^2 - s0 for any per-pixel constant s0; taking s0 close to the nearest
    // squared distance keeps the float32 rounding of t_i from being amplified
    // by a large d^2 (far field)
    const float s0 = sh > 0.0f ? 0.0f : (mine ? fmaxf(-log2f(d) / g.kappa, 0.0f) : 0.0f);
    if (lane < PS) {
      pxG[wid][lane] = make_float4(G[0], G[1], G[2], G[3]);
      pxQ[wid][lane] = make_float4(qx, qy, sp, emax);
      pxS[wid][lane] = make_float2(sh, s0);
    }
    const unsigned mm = __ballot_sync(full, mine);   // the micro-tile's non-core pixels
    float R2 = mine ? sh + emax : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) R2 = fmaxf(R2, __shfl_xor_sync(full, R2, o));
    R2 = R2 * (1.0f + 1e-6f) + 1e-6f;
    const float R = sqrtf(R2);
    const unsigned total = collect(a, g, t, R, R2, 0u, L);   // (ends with a warp sync: the pixels are in place)
    float sig = 0.0f;
    for (unsigned skip = 0; skip < total; skip += kFarCap) {
      if (skip > 0) collect(a, g, t, R, R2, skip, L);
      const unsigned n = min(total - skip, (unsigned)kFarCap);
      for (unsigned c0 = 0; c0 < n; c0 += 32) {
        const unsigned k = c0 + (unsigned)lane;
        const bool act = k < n;
        unsigned idx = 0;
        float2 p = make_float2(0.f, 0.f);
        float4 cv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (act) {
          idx = L[k];
          p = a.w.sxy[idx];
          cv = a.w.sval[idx];
        }
        const float c4[4] = {cv.x, cv.y, cv.z, cv.w};
        float cg[4] = {0.f, 0.f, 0.f, 0.f}, gx = 0.0f, gy = 0.0f;
        bool hit = false;   // some pixel keeps the pair
        for (unsigned rem = mm; rem; rem &= rem - 1u) {
          const int q = __ffs(rem) - 1;
          const float4 Gq = pxG[wid][q];
          const float4 Q = pxQ[wid][q];
          const float2 Sq = pxS[wid][q];
          const float dx = Q.x - p.x, dy = Q.y - p.y;
          const float ee = Sq.x > 0.0f ? shifted_sqdist(Q.x, Q.y, p.x, p.y, Sq.x) : fmaf(dx, dx, dy * dy);
          if (act && ee <= Q.w) {
            hit = true;
            const float w = ex2(-g.kappa * ee);
            const float Gv[4] = {Gq.x, Gq.y, Gq.z, Gq.w};
            float tt = -Q.z;
#pragma unroll
            for (int c = 0; c < C; ++c) tt = fmaf(Gv[c], c4[c], tt);
            const float wt = w * tt;
#pragma unroll
            for (int c = 0; c < C; ++c) cg[c] = fmaf(w, Gv[c], cg[c]);
            gx = fmaf(wt, dx, gx);
            gy = fmaf(wt, dy, gy);
            sig = fmaf(wt, ee - Sq.y, sig);   // ee is already d^2 - shift when shift > 0
          }
        }
        if (hit) {
          const unsigned o = a.w.perm[idx];
          if (bi.gvals) {
#pragma unroll
            for (int c = 0; c < C; ++c) atomicAdd(&bi.gvals[(long long)o * C + c], cg[c]);
          }
          if (bi.gpts) {
            atomicAdd(&bi.gpts[2LL * o], gx * bi.inv_s2);
            atomicAdd(&bi.gpts[2LL * o + 1], gy * bi.inv_s2);
          }
        }
      }
      __syncwarp();   // the list (and, after the last chunk, the pixels) are rewritten next
    }
    __syncwarp();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sig += __shfl_xor_sync(full, sig, o);
    if (lane == 0 && sig != 0.0f && bi.gsig) atomicAdd(bi.gsig, sig * bi.inv_s3);
  }
}

// Resident fallback blocks per SM (cached): the kernel is latency-bound, so
// its persistent grid fills every resident warp slot.
template <int C>
static int fallback_blocks_per_sm() {
  static const int n = [] {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, bwd_fallback_kernel<C>, 32 * kFarWarps, 0);
    return b > 0 ? b : 1;
  }();
  return n;
}

// The backward's region: per-pixel plane, fallback flags and queue, sigma
// partials, per-point moments, each 256-byte aligned and (checked builds)
// followed by a guard area.  sizes[] in bytes; returns the region's size.
static long long bwd_parts(long long N, int C, int H, int W, long long at[5], long long guard_at[5]) {
  const long long px = (long long)H * W;
  const long long mt = ((long long)H + 1) / 2 * (((long long)W + 3) / 4);   // smallest micro-tile: 2x4
  const long long sizes[5] = {px * 16 * (C == 4 ? 2 : 1), mt * 4, mt * 8, (long long)kSigParts * 4,
                              N * 4 * kPpMomentFloats};
  long long o = 0;
  for (int k = 0; k < 5; ++k) {
    at[k] = o;
    o += (sizes[k] + 255) / 256 * 256;
    guard_at[k] = o;
    o += (long long)kGuardBytes;
  }
  return o;
}

long long bwd_extra_bytes(long long N, int C, int H, int W) {
  long long at[5], ga[5];
  return bwd_parts(N, C, H, W, at, ga);
}

void bind_bwd(DevWork& w, void* extra, long long N, int C, int H, int W, long long mt_total) {
  (void)mt_total;
  long long at[5], ga[5];
  bwd_parts(N, C, H, W, at, ga);
  char* p = (char*)extra;
  w.pplane = (float4*)(p + at[0]);
  w.fbflag = (unsigned*)(p + at[1]);
  w.fbq = (uint2*)(p + at[2]);
  w.sig_part = (float*)(p + at[3]);
  w.ppmom = (float*)(p + at[4]);
}

void bwd_guards(long long N, int C, int H, int W, size_t extra_at, Guards& g) {
  if (kGuardBytes == 0) return;
  long long at[5], ga[5];
  bwd_parts(N, C, H, W, at, ga);
  for (int k = 0; k < 5 && g.n < kMaxGuards; ++k) g.off[g.n++] = extra_at + (size_t)ga[k];
}

template <int C>
static cudaError_t launch_bwd_c(const KArgs& a, const BwdArgs& b, cudaStream_t s) {
  const int sms = device_sm_count();
  const unsigned prep_blocks = (unsigned)std::max<long long>(1, std::min<long long>((a.px_total + 255) / 256, sms * 32LL));
  bwd_prep_kernel<C><<<prep_blocks, 256, 0, s>>>(a, b);
  const float rcore_log2 = kRelLog2 + kCoreLog2;   // kappa * R_core^2
  const unsigned blocks = (unsigned)std::max<long long>(1, std::min<long long>((a.n_total + 255) / 256, kSigParts));
  if (b.pp == 2) bwd_cov_kernel<C><<<blocks, 256, 0, s>>>(a, b);
  else if (b.pp) bwd_point_kernel<C, true, true><<<blocks, 256, 0, s>>>(a, b, rcore_log2);
  else if (b.trunc) bwd_point_kernel<C, true, false><<<blocks, 256, 0, s>>>(a, b, rcore_log2);
  else bwd_point_kernel<C, false, false><<<blocks, 256, 0, s>>>(a, b, rcore_log2);
  if (!b.trunc) bwd_fallback_kernel<C><<<sms * fallback_blocks_per_sm<C>(), 32 * kFarWarps, 0, s>>>(a, b);
  return cudaGetLastError();
}

cudaError_t launch_pp_exact_backward(const KArgs& a, const BwdImage& bi, int mth, int mtw, int ppk, float* mom,
                                     cudaStream_t s);

cudaError_t launch_backward(const KArgs& a, const BwdArgs& b, cudaStream_t s) {
  switch (a.C) {
    case 1: return launch_bwd_c<1>(a, b, s);
    case 2: return launch_bwd_c<2>(a, b, s);
    case 3: return launch_bwd_c<3>(a, b, s);
    default: return launch_bwd_c<4>(a, b, s);
  }
}

}  // namespace gmi

using namespace gmi;

// Backward pass with one shared sigma (sigmas == null: grad_sigma [1]) or
// per-point sigmas (grad_sigmas [N], shift may be null).
static gmi_status backward_impl(const float* points, const float* values, const float* sigmas, int64_t N, int C,
                                int H, int W, const gmi_params* p, const float* image, const float* den,
                                const float* shift, const float* grad_image, float* grad_points,
                                float* grad_values, float* grad_sigma, float* grad_sigmas, bool per_point,
                                int pp_kind, void* workspace, size_t ws_bytes, gmi_stream_t stream) {
  gmi_status st = check_params(p);
  if (st != GMI_OK) return st;
  if ((st = check_shape(N, C, H, W)) != GMI_OK) return st;
  if (!image || !den || (!shift && !per_point) || !grad_image || (N > 0 && (!points || !values)))
    return GMI_ERR_INVALID_ARG;
  if (((uintptr_t)points & 7u) != 0 || ((uintptr_t)values & 3u) != 0) return GMI_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int mth, mtw;
  variant_dims(p->variant, &mth, &mtw);
  ImageGeom g;
  memset(&g, 0, sizeof(g));
  fill_geom(g, N, H, W, p->sigma, p->radius_sigmas, p->bin_px, mth, mtw);
  g.points = points;
  g.values = values;
  g.sigmas = sigmas;
  g.pp_kind = sigmas ? pp_kind : 0;
  const long long nb = (long long)g.nbx * g.nby;
  const long long mt = (long long)g.mtx * g.mty;
  const long long wt = (long long)g.wtx * g.wty;
  const WsLayout L =
      ws_layout(N, nb, mt, wt, sat_entries(g), slot_bytes_for(mth, mtw, C), bwd_extra_bytes(N, C, H, W), true);
  if (!workspace || ((uintptr_t)workspace & 255u) != 0 || ws_bytes < L.total) return GMI_ERR_WORKSPACE;
  if (grad_points && cudaMemsetAsync(grad_points, 0, sizeof(float) * 2 * (size_t)N, s) != cudaSuccess) return GMI_ERR_CUDA;
  if (grad_values && cudaMemsetAsync(grad_values, 0, sizeof(float) * (size_t)C * (size_t)N, s) != cudaSuccess) return GMI_ERR_CUDA;
  if (grad_sigma && cudaMemsetAsync(grad_sigma, 0, sizeof(float), s) != cudaSuccess) return GMI_ERR_CUDA;
  if (grad_sigmas && cudaMemsetAsync(grad_sigmas, 0, sizeof(float) * (size_t)N * (size_t)pp_kind, s) != cudaSuccess)
    return GMI_ERR_CUDA;
  if (N == 0) return GMI_OK;

  KArgs a;
  memset(&a, 0, sizeof(a));
  a.w = bind_ws(workspace, L);
  bind_bwd(a.w, (char*)workspace + L.extra, N, C, H, W, mt);
  a.g0 = g;
  a.n_images = 1;
  a.C = C;
  a.n_total = N;
  a.nb_total = nb;
  a.wt_total = wt;
  a.ch_total = (N + kChunk - 1) / kChunk;
  a.mt_total = mt;
  a.satj_total = sat_jobs(g);
  const bool trunc = p->mode == GMI_MODE_TRUNCATED;
  if (kGuardBytes > 0) {
    Guards gx;
    gx.n = 0;
    bwd_guards(N, C, H, W, L.extra, gx);
    if (launch_canaries(workspace, gx, false, a.w.status, s) != cudaSuccess) return GMI_ERR_CUDA;
  }
  // the bins only: the fallback derives its radii from den, not from the plan
  if ((st = run_bin_and_plan(a, L, workspace, mth, mtw, trunc, s, false)) != GMI_OK) return st;
  if (per_point && !trunc) {
    // exact mode with per-point sigmas: every pixel's shift and den again,
    // the pairs' terms into per-point moments, then the gradients
    BwdImage bi;
    memset(&bi, 0, sizeof(bi));
    bi.grad = grad_image;
    bi.gpts = grad_points;
    bi.gvals = grad_values;
    bi.gsigs = grad_sigmas;
    const ProfileMark pm = profile_begin(GMI_STAGE_BACKWARD, s);
    if (launch_pp_exact_backward(a, bi, mth, mtw, g.pp_kind == 3 ? 2 : 1, a.w.ppmom, s) != cudaSuccess)
      return GMI_ERR_CUDA;
    profile_end(pm, s);
    return (p->flags & GMI_FLAG_SYNC_CHECK) ? read_status(workspace, s) : GMI_OK;
  }
  if (cudaMemsetAsync(a.w.fbflag, 0, sizeof(unsigned) * (size_t)mt, s) != cudaSuccess) return GMI_ERR_CUDA;
  a.px_total = (long long)H * W;
  BwdArgs b;
  memset(&b, 0, sizeof(b));
  b.one.image = image;
  b.one.den = den;
  b.one.shift = shift;
  b.one.grad = grad_image;
  b.one.gpts = grad_points;
  b.one.gvals = grad_values;
  b.one.gsig = grad_sigma;
  b.one.gsigs = grad_sigmas;
  b.one.inv_s2 = (float)(1.0 / ((double)p->sigma * p->sigma));
  b.one.inv_s3 = (float)(1.0 / ((double)p->sigma * p->sigma * p->sigma));
  b.table = nullptr;
  b.trunc = trunc ? 1 : 0;
  b.pp = g.pp_kind == 3 ? 2 : (g.pp_kind ? 1 : 0);
  const ProfileMark pm = profile_begin(GMI_STAGE_BACKWARD, s);
  if (launch_backward(a, b, s) != cudaSuccess) return GMI_ERR_CUDA;
  profile_end(pm, s);
  return (p->flags & GMI_FLAG_SYNC_CHECK) ? read_status(workspace, s) : GMI_OK;
}

extern "C" gmi_status gmi_backward(const float* points, const float* values, int64_t N, int C, int H, int W,
                                   const gmi_params* p, const float* image, const float* den, const float* shift,
                                   const float* grad_image, float* grad_points, float* grad_values,
                                   float* grad_sigma, void* workspace, size_t ws_bytes, gmi_stream_t stream) {
  return backward_impl(points, values, nullptr, N, C, H, W, p, image, den, shift, grad_image, grad_points,
                       grad_values, grad_sigma, nullptr, false, 0, workspace, ws_bytes, stream);
}

// Per-point sigmas: pp_kind floats per point, isotropic ([N]), axis-aligned
// ([N,2]) or a full covariance ([N,3]).
static gmi_status backward_per_point(const float* points, const float* values, const float* sigmas, int64_t N,
                                     int C, int H, int W, const gmi_params* p, const float* image,
                                     const float* den, const float* grad_image, float* grad_points,
                                     float* grad_values, float* grad_sigmas, int pp_kind, void* workspace,
                                     size_t ws_bytes, gmi_stream_t stream) {
  gmi_status st = check_params(p);
  if (st != GMI_OK) return st;
  if (N > 0 && (!sigmas || ((uintptr_t)sigmas & 3u) != 0)) return GMI_ERR_INVALID_ARG;
  return backward_impl(points, values, N > 0 ? sigmas : nullptr, N, C, H, W, p, image, den, nullptr, grad_image,
                       grad_points, grad_values, nullptr, grad_sigmas, true, pp_kind, workspace, ws_bytes, stream);
}

extern "C" gmi_status gmi_backward_pp(const float* points, const float* values, const float* sigmas, int64_t N,
                                      int C, int H, int W, const gmi_params* p, const float* image,
                                      const float* den, const float* grad_image, float* grad_points,
                                      float* grad_values, float* grad_sigmas, void* workspace, size_t ws_bytes,
                                      gmi_stream_t stream) {
  return backward_per_point(points, values, sigmas, N, C, H, W, p, image, den, grad_image, grad_points,
                            grad_values, grad_sigmas, 1, workspace, ws_bytes, stream);
}

extern "C" gmi_status gmi_backward_aniso(const float* points, const float* values, const float* sigmas_xy,
                                         int64_t N, int C, int H, int W, const gmi_params* p, const float* image,
                                         const float* den, const float* grad_image, float* grad_points,
                                         float* grad_values, float* grad_sigmas_xy, void* workspace,
                                         size_t ws_bytes, gmi_stream_t stream) {
  return backward_per_point(points, values, sigmas_xy, N, C, H, W, p, image, den, grad_image, grad_points,
                            grad_values, grad_sigmas_xy, 2, workspace, ws_bytes, stream);
}

extern "C" gmi_status gmi_backward_cov(const float* points, const float* values, const float* cov, int64_t N,
                                       int C, int H, int W, const gmi_params* p, const float* image,
                                       const float* den, const float* grad_image, float* grad_points,
                                       float* grad_values, float* grad_cov, void* workspace, size_t ws_bytes,
                                       gmi_stream_t stream) {
  return backward_per_point(points, values, cov, N, C, H, W, p, image, den, grad_image, grad_points, grad_values,
                            grad_cov, 3, workspace, ws_bytes, stream);
}
