// Near-field gather: the hot loop of the forward pass (Eq. 1 and Eq. 2).
//
// Each thread owns an MTH x MTW micro-tile of output pixels and keeps the
// numerators (C per pixel) and the denominator of Eq. 1 in registers.  The
// isotropic Gaussian factorises, 2^(-kappa d^2) = 2^(-kappa dx^2) 2^(-kappa dy^2),
// so one candidate point costs MTW + MTH exponentials (on the SFU) and
// (C + 1) fused multiply-adds per pixel: den += gy*gx, num_c += gy*(gx*c_c).
//
// Which points are candidates ("close enough", section 2): a pixel q needs
// every point with d^2 <= m_q + k^2 sigma^2, m_q being its squared distance
// to the nearest point; anything farther weighs less than e^{-k^2/2} of the
// nearest point.  The thread first bounds m_q from above for its pixels with
// the bin occupancy (a non-empty bin whose points all lie inside it contains
// a point no farther than its farthest corner), giving U >= max_q m_q, then
// sweeps every bin row that can hold a point within R = sqrt(U + k^2 sigma^2)
// of its pixels.  Bins are row-major sorted, so each bin row contributes one
// contiguous segment of the sorted point arrays.
//
// Range: weights are taken unshifted (no per-pixel subtraction of m_q), which
// is exact as long as every weight that matters stays a normal float:
// kappa * U <= 100 keeps the nearest weight >= 2^-100 and every weight within
// the radius >= 2^-126.  Micro-tiles that fail this (far from every point)
// are queued for the far-field kernel, which shifts per pixel.
//
// Load balance: a plan kernel estimates every warp tile's per-thread
// candidate count and cuts heavy tiles (dense clusters, wide sigma) into up to
// kSplitMax work items over each thread's candidate sequence; the items add
// their partial sums into one slot per tile (float reductions, so the order of
// those few additions varies from run to run) and the last one to finish
// writes the pixels.
//
// In truncated mode (the literal "radius k sigma" reading) R = k sigma, each
// pixel keeps only points with d^2 <= k^2 sigma^2, and nothing is queued.
//
// Per-point sigma (truncated mode only; PPK = 1: isotropic or axis-aligned):
// point i weighs 2^(la_i - kx_i dx^2 - ky_i dy^2) (pp_consts) and counts
// inside its ellipse kx_i dx^2 + ky_i dy^2 <= k^2 log2(e) / 2; the candidate
// window is that of the bound sigma >= sx_i, sy_i, and the factorisation is
// unchanged: gx = 2^(-kx_i dx^2), gy = 2^(la_i - ky_i dy^2).  PPK = 2, a full
// covariance (pp_cov_consts): the cross term kxy dx dy does not factorise,
// so every pixel takes its own exponential of
// la_i - (kxx dx^2 + kyy dy^2 + kxy dx dy), from per-column and per-row parts.
#include "bin_body.cuh"
#include "near_common.cuh"
#include "sat.cuh"

#include <algorithm>

namespace gmi {

int device_sm_count();

// Most bin rings searched for the nearest-distance bound.  A micro-tile whose
// nearest usable bin lies farther out goes to the far-field kernel, which
// finds its window with four-load summed-area-table counts instead of
// walking ring after ring bin by bin (measured: 16 rings -> 3 took the
// 64-image clustered batch from 1.374 to 1.310 ms and the 16 x 512^2
// clustered forward from 0.393 to 0.377 ms; 2 and 5 rings did no better).
constexpr int kRingMax = 3;

// Upper bound on max_q m_q over the micro-tile's valid pixels from bin
// occupancy, searched ring by ring around the micro-tile's bins (ring 0 its
// own bins, ring 1 the full neighbourhood one bin wider, later rings only
// their perimeter) until every pixel has a usable bin; +inf when that takes
// more than kRingMax rings (the micro-tile then belongs to the far-field
// kernel).
template <int MTH, int MTW>
__device__ float near_bound(const KArgs& a, const ImageGeom& g, int x0, int y0, int nx, int ny) {
  const float bf = (float)g.b;
  const float xq0 = (float)x0 + 0.5f, yq0 = (float)y0 + 0.5f;
  const int bx0 = (int)(xq0 * g.inv_b), bx1 = (int)((xq0 + (float)(nx - 1)) * g.inv_b);
  const int by0 = (int)(yq0 * g.inv_b), by1 = (int)((yq0 + (float)(ny - 1)) * g.inv_b);
  float best[MTH][MTW];
#pragma unroll
  for (int r = 0; r < MTH; ++r)
#pragma unroll
    for (int j = 0; j < MTW; ++j) best[r][j] = (r < ny && j < nx) ? INFINITY : 0.0f;

  // folds the usable bins of row `by`, columns [xa, xb], into best[][]
  auto scan_row = [&](int by, int xa, int xb) {
    if (by < 0 || by >= g.nby) return;
    xa = max(xa, 0);
    xb = min(xb, g.nbx - 1);
    if (xa > xb) return;
    const long long rowb = g.bin_base + (long long)by * g.nbx;
    float cy[MTH];
#pragma unroll
    for (int r = 0; r < MTH; ++r) {
      const float q = yq0 + (float)r;
      const float d0 = q - (float)by * bf, d1 = q - (float)(by + 1) * bf;
      cy[r] = fmaxf(d0 * d0, d1 * d1);
    }
    auto fold = [&](int bx) {
#pragma unroll
      for (int j = 0; j < MTW; ++j) {
        const float q = xq0 + (float)j;
        const float d0 = q - (float)bx * bf, d1 = q - (float)(bx + 1) * bf;
        const float cx = fmaxf(d0 * d0, d1 * d1);
#pragma unroll
        for (int r = 0; r < MTH; ++r) best[r][j] = fminf(best[r][j], cx + cy[r]);
      }
    };
    unsigned prev = __ldg(&a.w.off[rowb + xa]);
    for (int bx = xa; bx <= xb; ++bx) {
      const unsigned nxt = __ldg(&a.w.off[rowb + bx + 1]);
      const bool usable = nxt > prev && __ldg(&a.w.oob[rowb + bx]) == 0;
      prev = nxt;
      if (usable) fold(bx);
    }
  };

  // ring 0: the micro-tile's own bins; in dense regions they bound every
  // pixel.  With bins of two or more pixels they are at most RR rows of RC
  // bins, and every offset and flag of the ring is loaded in one round before
  // any is folded; 1-px bins walk the rows.
  constexpr int RR = MTH / 2 + 1, RC = MTW / 2 + 1;
  if (by1 - by0 < RR && bx1 - bx0 < RC) {
    unsigned o[RR][RC + 1];
    unsigned char fl[RR][RC];
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      const bool rin = by0 + r <= by1;
      const long long rowb = g.bin_base + (long long)(by0 + r) * g.nbx + bx0;
#pragma unroll
      for (int c = 0; c <= RC; ++c) o[r][c] = (rin && bx0 + c <= bx1 + 1) ? __ldg(&a.w.off[rowb + c]) : 0u;
#pragma unroll
      for (int c = 0; c < RC; ++c) fl[r][c] = (rin && bx0 + c <= bx1) ? __ldg(&a.w.oob[rowb + c]) : (unsigned char)1;
    }
#pragma unroll
    for (int rb = 0; rb < RR; ++rb) {
      if (by0 + rb > by1) break;
      const int by = by0 + rb;
      float cy[MTH];
#pragma unroll
      for (int r = 0; r < MTH; ++r) {
        const float q = yq0 + (float)r;
        const float d0 = q - (float)by * bf, d1 = q - (float)(by + 1) * bf;
        cy[r] = fmaxf(d0 * d0, d1 * d1);
      }
#pragma unroll
      for (int c = 0; c < RC; ++c) {
        if (bx0 + c > bx1) break;
        if (!(o[rb][c + 1] > o[rb][c] && fl[rb][c] == 0)) continue;
        const int bx = bx0 + c;
#pragma unroll
        for (int j = 0; j < MTW; ++j) {
          const float q = xq0 + (float)j;
          const float d0 = q - (float)bx * bf, d1 = q - (float)(bx + 1) * bf;
          const float cx = fmaxf(d0 * d0, d1 * d1);
#pragma unroll
          for (int r = 0; r < MTH; ++r) best[r][j] = fminf(best[r][j], cx + cy[r]);
        }
      }
    }
  } else {
    for (int by = by0; by <= by1; ++by) scan_row(by, bx0, bx1);
  }
  {
    float u = 0.0f;
#pragma unroll
    for (int r = 0; r < MTH; ++r)
#pragma unroll
      for (int j = 0; j < MTW; ++j) u = fmaxf(u, best[r][j]);
    if (u < INFINITY) return u;
  }
  for (int ring = 1; ring <= kRingMax; ++ring) {
    const int xa = bx0 - ring, xb = bx1 + ring;
    if (ring >= 2) {
      // points on this ring at all?  one row-segment count per side (independent
      // loads), so empty rings cost no per-bin work
      const int ca = max(xa, 0), cb = min(xb, g.nbx - 1);
      unsigned on_ring = 0;
      if (by0 - ring >= 0) {
        const long long rowb = g.bin_base + (long long)(by0 - ring) * g.nbx;
        on_ring += __ldg(&a.w.off[rowb + cb + 1]) - __ldg(&a.w.off[rowb + ca]);
      }
      if (by1 + ring < g.nby) {
        const long long rowb = g.bin_base + (long long)(by1 + ring) * g.nbx;
        on_ring += __ldg(&a.w.off[rowb + cb + 1]) - __ldg(&a.w.off[rowb + ca]);
      }
      const int ya = max(by0 - ring + 1, 0), yb = min(by1 + ring - 1, g.nby - 1);
#pragma unroll 4
      for (int by = ya; by <= yb; ++by) {
        const long long rowb = g.bin_base + (long long)by * g.nbx;
        if (xa >= 0) on_ring += __ldg(&a.w.off[rowb + xa + 1]) - __ldg(&a.w.off[rowb + xa]);
        if (xb < g.nbx) on_ring += __ldg(&a.w.off[rowb + xb + 1]) - __ldg(&a.w.off[rowb + xb]);
      }
      if (on_ring == 0) continue;
    }
    if (ring == 1) {
      for (int by = by0 - 1; by <= by1 + 1; ++by) scan_row(by, xa, xb);
    } else {
      scan_row(by0 - ring, xa, xb);
      scan_row(by1 + ring, xa, xb);
      for (int by = by0 - ring + 1; by <= by1 + ring - 1; ++by) {
        scan_row(by, xa, xa);
        scan_row(by, xb, xb);
      }
    }
    float u = 0.0f;
#pragma unroll
    for (int r = 0; r < MTH; ++r)
#pragma unroll
      for (int j = 0; j < MTW; ++j) u = fmaxf(u, best[r][j]);
    if (u < INFINITY) return u;
  }
  return INFINITY;
}

// What the plan loads for one warp tile in a single round: every thread's
// window row segments (its first kPassRows bin rows) and, for the staged
// gather, the warp window's union rows (lane r: row r).
struct PlanLoads {
  LaneWin w;
  unsigned segs[kPassRows], sege[kPassRows];   // this thread's rows: [start, end) of the sorted arrays
  unsigned S0, E0;                             // union row `lane`
  int wy_lo, rows;                             // the warp window's bin rows
};

template <int MTH, int MTW>
__device__ __forceinline__ void plan_loads(const KArgs& a, const ImageGeom& g, long long wt, bool act, float R2,
                                           int x0, int y0, int nx, int ny, PlanLoads& P) {
  const int lane = threadIdx.x & 31;
  int my_lo = INT_MAX, my_hi = INT_MIN;
  P.w.by_lo = 0;
  P.w.by_hi = -1;
  if (act) {
    P.w = lane_window(g, x0, y0, nx, ny, R2);
    my_lo = P.w.by_lo;
    my_hi = P.w.by_hi;
  }
  P.wy_lo = warp_min(my_lo);
  const int wy_hi = warp_max(my_hi);
  P.rows = wy_hi >= P.wy_lo ? wy_hi - P.wy_lo + 1 : 0;
  P.S0 = P.E0 = 0u;
  if (a.w.tplan && P.rows > 0 && P.rows <= kPassRows) {
    // the warp tile's pixel rectangle (clipped to the image) with the largest
    // radius of its threads: a superset of every thread's segment per row
    const float R2w = warp_maxf(act ? R2 : 0.0f);
    const unsigned lt = (unsigned)(wt - g.wt_base);
    const int X0 = (int)(lt % (unsigned)g.wtx) * 8 * MTW, Y0 = (int)(lt / (unsigned)g.wtx) * 4 * MTH;
    const LaneWin ww = lane_window(g, X0, Y0, min(8 * MTW, g.W - X0), min(4 * MTH, g.H - Y0), R2w);
    if (lane < P.rows) {
      int bxw_lo, bxw_hi;
      float hxw;
      row_bins(g, ww, P.wy_lo + lane, bxw_lo, bxw_hi, hxw);
      const long long rowb = g.bin_base + (long long)(P.wy_lo + lane) * g.nbx;
      P.S0 = __ldg(&a.w.off[rowb + bxw_lo]);
      P.E0 = __ldg(&a.w.off[rowb + bxw_hi + 1]);
    }
  }
#pragma unroll
  for (int k = 0; k < kPassRows; ++k) {
    P.segs[k] = P.sege[k] = 0u;
    if (act && P.w.by_lo + k <= P.w.by_hi) row_segment(a, g, P.w, P.w.by_lo + k, P.segs[k], P.sege[k]);
  }
}

// The staged gather's plan for warp tile wt (its first work item), from the
// loads above: the window bin rows, each row's union segment over the warp's
// threads, its place in the warp's staging buffer, and each thread's
// non-empty segments as indices of the staged copy.  The gather then issues
// its bulk copies after one round of loads.  A split tile, or a window larger
// than the buffer, is marked invalid (the gather sets such items up itself).
// `act`: the thread's micro-tile takes part (in the image, not far field).
template <int MTH, int MTW>
__device__ void tile_stage_plan(const KArgs& a, long long wt, bool act, const PlanLoads& P, unsigned S) {
  constexpr int CAP = StageCap<MTH, MTW>::value;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  TilePlanRec* rec = a.w.tplan + wt;
  bool valid = S == 1 && P.rows > 0 && P.rows <= kPassRows;
  unsigned total = 0;
  if (valid) {
    // records [S0, E0) of row r widened to even indices (16-byte boundaries
    // for the position copies), placed one after the other
    const unsigned need = P.E0 > P.S0 ? ((P.E0 + 1u) & ~1u) - (P.S0 & ~1u) : 0u;
    unsigned incl = min(need, (unsigned)CAP + 1u);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned u = __shfl_up_sync(full, incl, o);
      if (lane >= o) incl += u;
    }
    total = __shfl_sync(full, incl, 31);
    valid = total <= (unsigned)CAP;
    if (valid) {
      const unsigned abase = incl - need;
      const unsigned B = abase + (P.S0 & 1u);   // staged index of record S0
      unsigned nseg = 0;
#pragma unroll
      for (int k = 0; k < kPassRows; ++k) {
        const bool v = act && P.w.by_lo + k <= P.w.by_hi;
        const int r = v ? P.w.by_lo + k - P.wy_lo : 0;
        const unsigned Sr = __shfl_sync(full, P.S0, r), Br = __shfl_sync(full, B, r);
        const unsigned i0 = Br + (P.segs[k] - Sr), i1 = i0 + (P.sege[k] - P.segs[k]);
        if (v && i0 < i1) rec->seg[nseg++][lane] = i0 | (i1 << 16);
      }
      rec->lane[lane] = nseg | (act ? 0x80000000u : 0u);
      if (lane < P.rows) rec->rowc[lane] = make_uint2(P.S0 & ~1u, need | (abase << 16));
    }
  }
  if (lane == 0) rec->hdr = make_uint4((unsigned)P.rows | (valid ? 0x80000000u : 0u), total, (unsigned)P.wy_lo, 0u);
}

// Plan: one warp per warp tile.  Each thread bounds the nearest squared
// distance U of its micro-tile once (stored for the gather), queues far-field
// micro-tiles for the far kernel, and counts its candidates within
// R = sqrt(U + k^2 sigma^2); the tile is cut into S = ceil(max / kSplitTarget)
// work items, so that no single thread walks thousands of candidates while
// the rest of the GPU idles.  The count and the staging plan come from one
// round of loads.
template <int MTH, int MTW>
__device__ void near_plan_body(const KArgs& a, int trunc, long long wt) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  if (wt >= a.wt_total) return;
  const int img = find_image<1>(a, wt);
  const ImageGeom g = a.w.table ? a.w.table[img] : a.g0;
  const long long lt = wt - g.wt_base;
  const int mt_x = (int)((unsigned)lt % (unsigned)g.wtx) * 8 + (lane & 7);
  const int mt_y = (int)((unsigned)lt / (unsigned)g.wtx) * 4 + (lane >> 3);
  const int x0 = mt_x * MTW, y0 = mt_y * MTH;
  const bool active = x0 < g.W && y0 < g.H;
  const int nx = active ? min(MTW, g.W - x0) : 0;
  const int ny = active ? min(MTH, g.H - y0) : 0;
  // Bin offsets left invalid by a scan that gave up (ST_BINS; the load
  // overlaps near_bound's): the micro-tiles are then all marked inactive, no
  // far-field work is queued and no staging plan is valid, so that the
  // gathers after this kernel have nothing to walk (every read above stays
  // inside its array whatever the offsets hold).
  const bool bins_bad = bins_invalid(a.w.status);
  float U = 0.0f;
  bool far = false;
  if (!trunc && active) {
    U = near_bound<MTH, MTW>(a, g, x0, y0, nx, ny);
    far = !(U <= g.u_near_max);
  }
  if (bins_bad) {
    U = INFINITY;
    far = false;
  }
  if (!trunc) {
    const unsigned fm = __ballot_sync(full, far);
    if (fm) {
      const int leader = __ffs(fm) - 1;
      unsigned base = 0;
      if (lane == leader) base = atomicAdd(&a.w.status[kFarCount], (unsigned)__popc(fm));
      base = __shfl_sync(full, base, leader);
      const unsigned q = base + __popc(fm & ((1u << lane) - 1u));
      if (far && GMI_IN_BOUNDS(a.w, q, a.mt_total, CK_FARQ))
        a.w.farq[q] = make_uint2((unsigned)img, (unsigned)(mt_y * g.mtx + mt_x));
    }
  }
  a.w.ubound[wt * 32 + lane] = far ? INFINITY : U;
  const bool act = active && !far && !bins_bad;
  PlanLoads P;
  plan_loads<MTH, MTW>(a, g, wt, act, U + g.r2k, x0, y0, nx, ny, P);
  unsigned cnt = 0;
#pragma unroll
  for (int k = 0; k < kPassRows; ++k) cnt += P.sege[k] - P.segs[k];
  if (act) {
    // rows past the first kPassRows (wide windows)
    for (int by = P.w.by_lo + kPassRows; by <= P.w.by_hi; ++by) {
      unsigned s0, e0;
      row_segment(a, g, P.w, by, s0, e0);
      cnt += e0 - s0;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt = max(cnt, __shfl_xor_sync(full, cnt, o));
  // small problems: finer items, so that there are about as many items as
  // resident warps (latency hiding needs several warps per scheduler)
  const unsigned target = (unsigned)max(48LL, min((long long)kSplitTarget, (long long)kSplitTarget * a.wt_total / 2368));
  unsigned S = min((cnt + target - 1) / target, (unsigned)kSplitMax);
  if (S < 1) S = 1;
  unsigned slot = 0xffffffffu;
  if (S > 1) {
    // one accumulation slot per split tile, zeroed here; its items add into it
    if (lane == 0) slot = atomicAdd(&a.w.status[kSlotCount], 1u);
    slot = __shfl_sync(full, slot, 0);
    if (slot >= a.cap_slots) {   // cannot happen (one slot per warp tile); keep the tile whole
      S = 1;
      slot = 0xffffffffu;
    } else {
      const int na = a.mth * a.mtw * (a.C + 1);
      float4* z = reinterpret_cast<float4*>(a.w.slots + ((size_t)slot * 32 + lane) * na);
      for (int k = 0; k < na / 4; ++k) z[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  if (a.w.tplan) tile_stage_plan<MTH, MTW>(a, wt, act, P, S);
  // the tile's first item sits at index wt (so a near-kernel warp can start on
  // warp tile t without reading the queue first); its other splits follow
  // all first items
  if (lane == 0) {
    a.w.items[wt] = make_uint4((unsigned)wt, S << 16, slot, (unsigned)img);
    if (S > 1) {
      const unsigned long long base = (unsigned long long)a.wt_total + atomicAdd(&a.w.status[kItemCount], S - 1);
      for (unsigned k = 1; k < S && base + k - 1 < a.cap_items; ++k)
        a.w.items[base + k - 1] = make_uint4((unsigned)wt, k | (S << 16), slot, (unsigned)img);
    }
  }
}

// Plan (blocks [0, n_plan), one warp per warp tile) and scatter (the
// remaining n_scatter blocks) in one launch: the plan needs only the bin
// offsets and flags, which the scan has already produced, so the two run side
// by side.  The plan's warps are latency-bound chains of small loads, so they
// get the low block indices and start first; the scatter streams around them.
// STRIDE (batched calls, whose grids follow the plan's capacity, often far
// above the batch's warp tiles): fewer plan blocks, their warps striding over
// the warp tiles.
template <int MTH, int MTW, bool STRIDE>
__global__ void __launch_bounds__(256, 3) scatter_plan_kernel(KArgs a_in, int trunc, int n_scatter, int n_plan) {
  const KArgs a = resolve(a_in);
  if ((int)blockIdx.x < n_plan) {
    const long long wt0 = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (STRIDE) {
      for (long long wt = wt0; wt < a.wt_total; wt += (long long)n_plan * 8) near_plan_body<MTH, MTW>(a, trunc, wt);
    } else {
      near_plan_body<MTH, MTW>(a, trunc, wt0);
    }
  } else {
    bin_scatter_body(a, n_scatter, (int)blockIdx.x - n_plan);
  }
}

// Resident 128-thread blocks per SM the register budget is sized for, from
// the accumulators a thread holds (MTH * MTW pixels times C + 1 sums).
template <int MTH, int MTW, int C>
struct NearOcc {
  static constexpr int acc = MTH * MTW * (C + 1);
  static constexpr int value = acc <= 32 ? 5 : (acc <= 64 ? 4 : (acc <= 80 ? 3 : 2));
};

constexpr int kNearWarps = 4;   // warps per near-kernel block

template <int MTH, int MTW, int C, bool TRUNC, int PPK>
__global__ void __launch_bounds__(128, NearOcc<MTH, MTW, C>::value) near_kernel(KArgs a_in) {
  constexpr bool PP = PPK != 0;   // per-point sigmas (1: separable, 2: full covariance)
  static_assert(TRUNC || !PP, "per-point sigma is built for truncated mode only");
  const KArgs a = resolve(a_in);
  constexpr int NA = MTH * MTW * (C + 1);   // accumulators per thread
  constexpr int NP = (C + 1) / 2;           // packed accumulator pairs per pixel
  constexpr int ODD = (C + 1) & 1;          // one scalar accumulator left over (C even)
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int lx = lane & 7, ly = lane >> 3;
  const int warp = threadIdx.x >> 5;

  const unsigned n_items = (unsigned)min((unsigned long long)a.wt_total + a.w.status[kItemCount],
                                         (unsigned long long)a.cap_items);
  const unsigned n_warps = gridDim.x * kNearWarps;
  // first item by warp index, later ones claimed from the queue (the claim is
  // made once the item's sums are complete, so that its latency overlaps the
  // stores without holding an item while this one is still being computed)
  unsigned t = blockIdx.x * kNearWarps + warp;
  while (t < n_items) {
    const uint4 item = a.w.items[t];
    const long long wt = (long long)item.x;
    const unsigned split = item.y & 0xffffu, S = item.y >> 16, slot = item.z;
    const int img = (int)item.w;
    const ImageGeom g = a.w.table ? a.w.table[img] : a.g0;
    const long long lt = wt - g.wt_base;
    const int mt_x = (int)((unsigned)lt % (unsigned)g.wtx) * 8 + lx;
    const int mt_y = (int)((unsigned)lt / (unsigned)g.wtx) * 4 + ly;
    const int x0 = mt_x * MTW, y0 = mt_y * MTH;
    bool active = x0 < g.W && y0 < g.H;
    const int nx = active ? min(MTW, g.W - x0) : 0;
    const int ny = active ? min(MTH, g.H - y0) : 0;

    float R2 = g.r2k;
    if (!TRUNC) {
      // bound from the plan; +inf marks a far-field micro-tile (queued there)
      const float U = __ldcg(&a.w.ubound[wt * 32 + lane]);
      if (!(U <= g.u_near_max)) active = false;
      R2 = U + g.r2k;
    }

    // Accumulators in packed pairs (FFMA2 updates two per instruction): per
    // pixel (r, j) the pairs (den, num_0), (num_1, num_2), plus num_{C-1}
    // alone when C is even.
    float2 accp[MTH * MTW * NP];
    float accs[MTH * MTW * ODD + 1 - ODD];
#pragma unroll
    for (int k = 0; k < MTH * MTW * NP; ++k) accp[k] = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < MTH * MTW * ODD + 1 - ODD; ++k) accs[k] = 0.0f;

    // one candidate point (position p, colour cv, per-point sigma constants
    // spc when PP) into every pixel of the micro-tile
    // truncated mode: keep -kappa d^2 >= this
    const float neg_thr = PP ? -g.e_trunc : -g.kappa * g.r2k;
    const float xq0 = (float)x0 + 0.5f, yq0 = (float)y0 + 0.5f;
    auto consume = [&](const float2 p, const float4 cv, const float4 spc) {
      const float sk = PP ? spc.x : g.sk;     // along x
      const float sky = PP ? spc.y : g.sk;    // along y
      const float c4[4] = {cv.x, cv.y, cv.z, cv.w};
      float2 cp[NP];   // (1, c_0), (c_1, c_2)
      cp[0] = make_float2(1.0f, c4[0]);
#pragma unroll
      for (int q = 1; q < NP; ++q) cp[q] = make_float2(c4[2 * q - 1], c4[2 * q]);
      const float clast = c4[C - 1];   // the scalar accumulator's value (C even)
      if constexpr (PPK == 2) {
        // full covariance: e = -(kxx dx^2 + kyy dy^2 + kxy dx dy) per pixel
        const float dx0 = xq0 - p.x, dy0 = yq0 - p.y;
        float dx[MTW], ax[MTW], ay[MTH], by[MTH];
#pragma unroll
        for (int j = 0; j < MTW; ++j) {
          dx[j] = __fadd_rn(dx0, (float)j);
          ax[j] = __fmul_rn(-__fmul_rn(spc.x, dx[j]), dx[j]);
        }
#pragma unroll
        for (int r = 0; r < MTH; ++r) {
          const float dy = __fadd_rn(dy0, (float)r);
          ay[r] = __fmul_rn(-__fmul_rn(spc.z, dy), dy);
          by[r] = __fmul_rn(-spc.y, dy);
        }
#pragma unroll
        for (int r = 0; r < MTH; ++r)
#pragma unroll
          for (int j = 0; j < MTW; ++j) {
            const float e = __fmaf_rn(by[r], dx[j], __fadd_rn(ax[j], ay[r]));
            const float wgt = e >= neg_thr ? ex2(__fadd_rn(e, spc.w)) : 0.0f;
            const float2 ww = make_float2(wgt, wgt);
#pragma unroll
            for (int q = 0; q < NP; ++q) {
              float2& acq = accp[(r * MTW + j) * NP + q];
              acq = __ffma2_rn(ww, cp[q], acq);
            }
            if (ODD) accs[(r * MTW + j) * ODD] = fmaf(wgt, clast, accs[(r * MTW + j) * ODD]);
          }
        return;
      }
      const float u = (xq0 - p.x) * sk;
      const float v = (yq0 - p.y) * sky;
      float ax[MTW], gx[MTW], ay[MTH], gy[MTH];
      // (per-point sigma: explicit roundings, which the backward pass repeats
      // to keep exactly the same pairs)
#pragma unroll
      for (int j = 0; j < MTW; ++j) {
        const float tt = PP ? __fmaf_rn((float)j, sk, u) : u + (float)j * sk;
        ax[j] = PP ? __fmul_rn(-tt, tt) : -tt * tt;
        gx[j] = ex2(ax[j]);
      }
#pragma unroll
      for (int r = 0; r < MTH; ++r) {
        const float tt = PP ? __fmaf_rn((float)r, sky, v) : v + (float)r * sky;
        ay[r] = PP ? __fmul_rn(-tt, tt) : -tt * tt;
        gy[r] = ex2(PP ? __fadd_rn(ay[r], spc.z) : ay[r]);
      }
      if (!TRUNC) {
        // separable weight gy[r] * gx[j]: the column factors times the
        // point's values once, then one FFMA2 per pair and pixel (the first
        // pair (gx, gx c_0) is one scalar product: its other half is gx * 1)
        float2 hx[MTW][NP];
        float hs[MTW];
#pragma unroll
        for (int j = 0; j < MTW; ++j) {
#pragma unroll
          for (int q = 0; q < NP; ++q)
            hx[j][q] = q == 0 ? make_float2(gx[j], gx[j] * cp[0].y) : __fmul2_rn(make_float2(gx[j], gx[j]), cp[q]);
          if (ODD) hs[j] = gx[j] * clast;
        }
#pragma unroll
        for (int r = 0; r < MTH; ++r) {
          const float2 gg = make_float2(gy[r], gy[r]);
#pragma unroll
          for (int j = 0; j < MTW; ++j) {
#pragma unroll
            for (int q = 0; q < NP; ++q) {
              float2& acq = accp[(r * MTW + j) * NP + q];
              acq = __ffma2_rn(gg, hx[j][q], acq);
            }
            if (ODD) accs[(r * MTW + j) * ODD] = fmaf(gy[r], hs[j], accs[(r * MTW + j) * ODD]);
          }
        }
      } else {
#pragma unroll
        for (int r = 0; r < MTH; ++r)
#pragma unroll
          for (int j = 0; j < MTW; ++j) {
            const float e = PP ? __fadd_rn(ax[j], ay[r]) : ax[j] + ay[r];
            const float wgt = (e >= neg_thr) ? gx[j] * gy[r] : 0.0f;
            const float2 ww = make_float2(wgt, wgt);
#pragma unroll
            for (int q = 0; q < NP; ++q) {
              float2& acq = accp[(r * MTW + j) * NP + q];
              acq = __ffma2_rn(ww, cp[q], acq);
            }
            if (ODD) accs[(r * MTW + j) * ODD] = fmaf(wgt, clast, accs[(r * MTW + j) * ODD]);
          }
      }
    };

    if (active) {
      const LaneWin w = lane_window(g, x0, y0, nx, ny, R2);
      unsigned lo, hi;
      item_share(a, g, w, split, S, lo, hi);
      direct_walk<PP>(a, g, w, lo, hi, consume);
    }

    unsigned nt = n_items;   // (no claim when the items do not outnumber the warps)
    if (lane == 0 && n_items > n_warps) nt = n_warps + atomicAdd(&a.w.status[kNearHead], 1u);

    float acc[NA];   // per pixel (r, j): [den, num_0 .. num_{C-1}]
#pragma unroll
    for (int px = 0; px < MTH * MTW; ++px)
#pragma unroll
      for (int k = 0; k <= C; ++k) {
        if (k < 2 * NP) {
          const float2 pr = accp[px * NP + k / 2];
          acc[px * (C + 1) + k] = (k & 1) ? pr.y : pr.x;
        } else {
          acc[px * (C + 1) + k] = accs[px * ODD];
        }
      }

    bool finish = true;
    if (S > 1 && GMI_IN_BOUNDS(a.w, slot, a.cap_slots, CK_SLOT)) {
      // split tile: add this item's partial sums into the tile's slot; the
      // last item to finish reads the totals and writes the pixels
      float* mine = a.w.slots + ((size_t)slot * 32 + lane) * NA;
      if (active) {
#pragma unroll
        for (int k = 0; k < NA; k += 4)
          asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(mine + k), "f"(acc[k]),
                       "f"(acc[k + 1]), "f"(acc[k + 2]), "f"(acc[k + 3])
                       : "memory");
      }
      __threadfence();
      __syncwarp();
      unsigned prev = 0;
      if (lane == 0) prev = atomicAdd(&a.w.tile_done[wt], 1u);
      prev = __shfl_sync(full, prev, 0);
      finish = prev == S - 1;
      if (finish) {
        __threadfence();
        if (active) {
#pragma unroll
          for (int k = 0; k < NA; k += 4) {
            const float4 v = __ldcg(reinterpret_cast<const float4*>(mine + k));
            acc[k] = v.x;
            acc[k + 1] = v.y;
            acc[k + 2] = v.z;
            acc[k + 3] = v.w;
          }
        }
      }
    }
    if (finish && active) {
      // normalise (Eq. 1) and store
#pragma unroll
      for (int r = 0; r < MTH; ++r) {
        if (r >= ny) break;
        float outv[MTW * C];
        float denv[MTW];
#pragma unroll
        for (int j = 0; j < MTW; ++j) {
          const float* q = acc + (r * MTW + j) * (C + 1);
          const float d = q[0];
          const float inv = d > 0.0f ? __frcp_rn(d) : 0.0f;   // = 1 / d, correctly rounded
          denv[j] = d;
#pragma unroll
          for (int ch = 0; ch < C; ++ch) outv[j * C + ch] = q[1 + ch] * inv;
        }
        const long long row = (long long)(y0 + r) * g.W + x0;
        if (MTW % 4 == 0 && g.vec_ok && nx == MTW) {   // rows of whole float4s
          float4* o = reinterpret_cast<float4*>(g.image + row * C);
#pragma unroll
          for (int k = 0; k < MTW * C / 4; ++k) o[k] = make_float4(outv[4 * k], outv[4 * k + 1], outv[4 * k + 2], outv[4 * k + 3]);
          if (g.den) {
            float4* dd = reinterpret_cast<float4*>(g.den + row);
#pragma unroll
            for (int k = 0; k < MTW / 4; ++k) dd[k] = make_float4(denv[4 * k], denv[4 * k + 1], denv[4 * k + 2], denv[4 * k + 3]);
          }
          if (g.shift) {
            float4* ss = reinterpret_cast<float4*>(g.shift + row);
#pragma unroll
            for (int k = 0; k < MTW / 4; ++k) ss[k] = make_float4(0.f, 0.f, 0.f, 0.f);
          }
        } else {
#pragma unroll
          for (int j = 0; j < MTW; ++j) {
            if (j >= nx) break;
#pragma unroll
            for (int ch = 0; ch < C; ++ch) g.image[(row + j) * C + ch] = outv[j * C + ch];
            if (g.den) g.den[row + j] = denv[j];
            if (g.shift) g.shift[row + j] = 0.0f;
          }
        }
      }
    }
    t = __shfl_sync(full, nt, 0);
  }
  // far-field micro-tiles queued: warps out of work build the summed-area
  // table the far kernel's window search reads
  if constexpr (!TRUNC) {
    if (__ldcg(&a.w.status[kFarCount]) > 0u) sat_build(a);
  }
}

// Resident blocks per SM of one near-kernel instantiation (register-limited,
// as the launch bounds ask), cached; all devices of a process are taken to be alike.
template <int MTH, int MTW, int C, bool TRUNC, int PPK>
static int near_occ() {
  static const int n = [] {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, near_kernel<MTH, MTW, C, TRUNC, PPK>, 32 * kNearWarps, 0);
    return b > 0 ? b : 1;
  }();
  return n;
}

template <int MTH, int MTW, int C, bool TRUNC, int PPK>
static cudaError_t launch_near_k(const KArgs& a, int grid, cudaStream_t s) {
  near_kernel<MTH, MTW, C, TRUNC, PPK><<<grid, 32 * kNearWarps, 0, s>>>(a);
  return cudaGetLastError();
}

// mode: 0 exact, 1 truncated, 2 truncated with separable per-point sigmas,
// 3 truncated with a full covariance per point
template <int MTH, int MTW, int C>
static cudaError_t launch_near_c(const KArgs& a, int mode, int grid, cudaStream_t s) {
  switch (mode) {
    case 0: return launch_near_k<MTH, MTW, C, false, 0>(a, grid, s);
    case 1: return launch_near_k<MTH, MTW, C, true, 0>(a, grid, s);
    case 2: return launch_near_k<MTH, MTW, C, true, 1>(a, grid, s);
    default: return launch_near_k<MTH, MTW, C, true, 2>(a, grid, s);
  }
}

template <int MTH, int MTW>
static cudaError_t launch_near_mt(const KArgs& a, int mode, int grid, cudaStream_t s) {
  switch (a.C) {
    case 1: return launch_near_c<MTH, MTW, 1>(a, mode, grid, s);
    case 2: return launch_near_c<MTH, MTW, 2>(a, mode, grid, s);
    case 3: return launch_near_c<MTH, MTW, 3>(a, mode, grid, s);
    default: return launch_near_c<MTH, MTW, 4>(a, mode, grid, s);
  }
}

// Resident 256-thread blocks of the fused scatter + plan kernel on the whole
// device (the 4 x 4 instantiation stands for all: they share the register
// bound), cached.
static int scatter_plan_slots() {
  static const int n = [] {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, scatter_plan_kernel<4, 4, false>, 256, 0) != cudaSuccess ||
        b < 1)
      b = 1;
    return b * device_sm_count();
  }();
  return n;
}

void warm_scatter_plan() { scatter_plan_slots(); }

// n_scatter scatter blocks (0: scatter not needed) followed by the plan's blocks.
cudaError_t launch_scatter_plan(const KArgs& a, bool trunc, int n_scatter, cudaStream_t s) {
  // one block per 8 warp tiles; batched (capacity-sized): at most 64 blocks
  // per SM, the warps striding
  const bool stride = a.totals != nullptr;
  const long long need = (a.wt_total + 7) / 8;
  const int n_plan = (int)(stride ? std::min<long long>(need, 64LL * device_sm_count()) : need);
  if (!stride && n_scatter > 0) {
    // single image: the scatter's blocks take the resident slots the plan's
    // blocks leave free (one wave), each looping over its chunks; the plan's
    // blocks, the longer chains, then never wait for a slot
    const int slots = scatter_plan_slots();
    n_scatter = std::min(n_scatter, std::max(device_sm_count(), slots - n_plan));
  }
  const unsigned blocks = (unsigned)(n_scatter + n_plan);
  const int t = trunc ? 1 : 0;
  if (stride) {
    if (a.mth == 4 && a.mtw == 8) scatter_plan_kernel<4, 8, true><<<blocks, 256, 0, s>>>(a, t, n_scatter, n_plan);
    else if (a.mth == 2 && a.mtw == 4) scatter_plan_kernel<2, 4, true><<<blocks, 256, 0, s>>>(a, t, n_scatter, n_plan);
    else if (a.mth == 4 && a.mtw == 2) scatter_plan_kernel<4, 2, true><<<blocks, 256, 0, s>>>(a, t, n_scatter, n_plan);
    else scatter_plan_kernel<4, 4, true><<<blocks, 256, 0, s>>>(a, t, n_scatter, n_plan);
  } else {
    if (a.mth == 4 && a.mtw == 8) scatter_plan_kernel<4, 8, false><<<blocks, 256, 0, s>>>(a, t, n_scatter, n_plan);
    else if (a.mth == 2 && a.mtw == 4) scatter_plan_kernel<2, 4, false><<<blocks, 256, 0, s>>>(a, t, n_scatter, n_plan);
    else if (a.mth == 4 && a.mtw == 2) scatter_plan_kernel<4, 2, false><<<blocks, 256, 0, s>>>(a, t, n_scatter, n_plan);
    else scatter_plan_kernel<4, 4, false><<<blocks, 256, 0, s>>>(a, t, n_scatter, n_plan);
  }
  return cudaGetLastError();
}

// ppk: 0 shared sigma, 1 separable per-point sigmas, 2 full covariance per point
static int near_mode(bool trunc, int ppk) { return ppk ? 1 + ppk : (trunc ? 1 : 0); }

cudaError_t launch_near(const KArgs& a, int mth, int mtw, bool trunc, int ppk, int grid, cudaStream_t s) {
  const int m = near_mode(trunc, ppk);
  if (mth == 4 && mtw == 4) return launch_near_mt<4, 4>(a, m, grid, s);
  if (mth == 4 && mtw == 8) return launch_near_mt<4, 8>(a, m, grid, s);
  if (mth == 2 && mtw == 4) return launch_near_mt<2, 4>(a, m, grid, s);
  if (mth == 4 && mtw == 2) return launch_near_mt<4, 2>(a, m, grid, s);
  return cudaErrorInvalidValue;
}

// Resident near-kernel blocks per SM for an instantiation (cached).
template <int MTH, int MTW, int C>
static int occ_c(int mode) {
  switch (mode) {
    case 0: return near_occ<MTH, MTW, C, false, 0>();
    case 1: return near_occ<MTH, MTW, C, true, 0>();
    case 2: return near_occ<MTH, MTW, C, true, 1>();
    default: return near_occ<MTH, MTW, C, true, 2>();
  }
}

template <int MTH, int MTW>
static int occ_mt(int C, int mode) {
  switch (C) {
    case 1: return occ_c<MTH, MTW, 1>(mode);
    case 2: return occ_c<MTH, MTW, 2>(mode);
    case 3: return occ_c<MTH, MTW, 3>(mode);
    default: return occ_c<MTH, MTW, 4>(mode);
  }
}

int near_blocks_per_sm(int mth, int mtw, int C, bool trunc, int ppk) {
  const int c = C < 1 ? 1 : (C > 4 ? 4 : C);
  const int m = near_mode(trunc, ppk);
  if (mth == 4 && mtw == 8) return occ_mt<4, 8>(c, m);
  if (mth == 2 && mtw == 4) return occ_mt<2, 4>(c, m);
  if (mth == 4 && mtw == 2) return occ_mt<4, 2>(c, m);
  return occ_mt<4, 4>(c, m);
}

}  // namespace gmi
