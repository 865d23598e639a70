// Bin key of a point and the scatter into bin-sorted arrays, shared by the
// binning kernels and the fused scatter + plan launch.
#pragma once

#include "common.cuh"

namespace gmi {

static __device__ __forceinline__ void point_bin(const ImageGeom& g, float x, float y, long long& bin,
                                          bool& oob) {
  int bx = bin_coord(x, g.inv_b, g.nbx);
  int by = bin_coord(y, g.inv_b, g.nby);
  bin = g.bin_base + (long long)by * g.nbx + bx;
  oob = !(x >= 0.0f && x < (float)g.W && y >= 0.0f && y < (float)g.H);
}

// Scatter of a single image with one shared sigma: the image's geometry
// read once, nothing but the copies per point.
static __device__ __forceinline__ void scatter_single(const KArgs& a, int nblocks, int block) {
  const ImageGeom g = a.g0;
  bool fin = true;
  for (long long ch = block; ch < a.ch_total; ch += nblocks) {
    const long long i = ch * kChunk + threadIdx.x;
    if (i < g.n) {
      const float2 p = reinterpret_cast<const float2*>(g.points)[i];
      long long bin;
      bool oob;
      point_bin(g, p.x, p.y, bin, oob);
      const unsigned dst = a.w.off[bin] + a.w.rank[i];
      float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
      const float* v = g.values + i * a.C;
      c.x = v[0];
      if (a.C > 1) c.y = v[1];
      if (a.C > 2) c.z = v[2];
      if (a.C > 3) c.w = v[3];
      fin = fin && isfinite(c.x) && isfinite(c.y) && isfinite(c.z) && isfinite(c.w);
      // (dst < n_total also when the scan gave up and the offsets are not valid)
      if (GMI_IN_BOUNDS(a.w, dst, a.n_total, CK_SCATTER) && dst < (unsigned long long)a.n_total) {
        a.w.sxy[dst] = p;
        a.w.sval[dst] = c;
        a.w.perm[dst] = (unsigned)i;
      }
    }
  }
  if (__any_sync(0xffffffffu, !fin) && (threadIdx.x & 31) == 0) atomicOr(&a.w.status[kStatusErr], ST_NONFINITE);
}

// Scatter body: `nblocks` blocks stride over the chunks; this block is number
// `block` of them.
static __device__ __forceinline__ void bin_scatter_body(const KArgs& a, int nblocks, int block) {
  if (!a.w.table && !a.g0.sigmas) {
    scatter_single(a, nblocks, block);
    return;
  }
  bool fin = true;
  for (long long ch = block; ch < a.ch_total; ch += nblocks) {
    const int img = find_image<0>(a, ch);
    const ImageGeom g = a.w.table ? a.w.table[img] : a.g0;   // a copy: no address of a local struct
    const long long i = (ch - g.ch_base) * kChunk + threadIdx.x;
    float la = 0.0f;   // this point's log2 normaliser (per-point sigmas)
    if (i < g.n) {
      float2 p = reinterpret_cast<const float2*>(g.points)[i];
      long long bin;
      bool oob;
      point_bin(g, p.x, p.y, bin, oob);
      unsigned dst = a.w.off[bin] + a.w.rank[g.pt_base + i];
      float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
      const float* v = g.values + i * a.C;
      c.x = v[0];
      if (a.C > 1) c.y = v[1];
      if (a.C > 2) c.z = v[2];
      if (a.C > 3) c.w = v[3];
      fin = fin && isfinite(c.x) && isfinite(c.y) && isfinite(c.z) && isfinite(c.w);
      const bool ok = GMI_IN_BOUNDS(a.w, dst, a.n_total, CK_SCATTER) && dst < (unsigned long long)a.n_total;
      if (ok) {
        a.w.sxy[dst] = p;
        a.w.sval[dst] = c;
        a.w.perm[dst] = (unsigned)i;
      }
      if (g.sigmas && ok) {
        const float* sg = g.sigmas + g.pp_kind * i;
        const float4 k = g.pp_kind == 3 ? pp_cov_consts(g.sigma, sg[0], sg[1], sg[2])
                                        : pp_consts(g.sigma, sg[0], g.pp_kind == 2 ? sg[1] : sg[0]);
        a.w.spp[dst] = k;
        la = g.pp_kind == 3 ? k.w : k.z;
      }
    }
    if (g.sigmas) {
      // the image's largest normaliser (exact mode's candidate radius): one
      // atomic per warp; la >= 0, so its bits order as the values do
      la = (la >= 0.0f && la < INFINITY) ? la : 0.0f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) la = fmaxf(la, __shfl_xor_sync(0xffffffffu, la, o));
      if ((threadIdx.x & 31) == 0) atomicMax(&a.w.status[kLaMax], __float_as_uint(la));
    }
  }
  if (__any_sync(0xffffffffu, !fin) && (threadIdx.x & 31) == 0) atomicOr(&a.w.status[kStatusErr], ST_NONFINITE);
}

}  // namespace gmi
