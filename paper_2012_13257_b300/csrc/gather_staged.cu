// Near-field gather with staged candidates: the forward pass's hot loop
// (Eq. 1 and Eq. 2 of section 2) for one shared sigma, exact or truncated.
//
// The arithmetic is that of the direct-load gather (gather_near.cu): each
// thread owns an MTH x MTW micro-tile of pixels, the isotropic weight
// factorises as 2^(-kappa dx^2) 2^(-kappa dy^2), and one candidate costs
// MTW + MTH exponentials on the SFU and C + 1 fused multiply-adds per pixel,
// accumulated in FP32 registers.  What differs is how the candidates reach
// the threads.
//
// A thread's candidates are the bin-row segments of the bin-sorted arrays
// within its radius (row_segment).  The warp stages the union of its threads'
// windows: lane r takes bin row r of the window and computes that row's
// segment for the whole warp tile with the largest radius (a superset of
// every thread's segment in the row, the window arithmetic being monotone);
// each row's positions and colours are then copied from global into shared
// memory with one bulk copy per array (cp.async.bulk on the TMA engine,
// completion counted in bytes on an mbarrier).  The bin offsets of the union
// rows and of every thread's own rows are loaded in one round trip, and each
// thread turns its own segments into indices of the staged copy.  The walk
// then reads shared memory only, neighbouring lanes reading neighbouring
// records.  (Trimming each segment's ends to the thread's x-extent in its
// row was measured: the trim loops cost more than the few records they skip.)
//
// A window with more records than the buffer holds (dense clusters, wide
// radii) is walked straight from global memory instead: each thread lists its
// row segments in the warp's (then unused) staging buffer and keeps its next
// few candidates in flight through a per-lane ring there (cp.async); a window
// with more bin rows than the list holds takes the row-by-row direct walk of
// near_common.cuh.  A heavy warp tile cut into S work items
// (the plan in gather_near.cu) gives item k the k-th share of every thread's
// candidate sequence.  Every wait on the barrier is bounded: if one gives up,
// the kernel sets ST_TIMEOUT in the status word, waits (bounded again) for
// its copies still in flight, and leaves.
#include "far_tile.cuh"
#include "near_common.cuh"
#include "sat.cuh"

#include <algorithm>
#include <climits>

namespace gmi {

constexpr int kStageWarps = 4;    // warps per block
// A barrier wait polls at most kWaitPolls times; each poll may suspend the
// thread for up to kWaitHintNs until the phase completes (so a wait gives up
// after about a second, and a waiting warp takes no issue slots meanwhile).
constexpr unsigned kWaitPolls = 10000u;
constexpr unsigned kWaitHintNs = 100000u;

// Polls of the first wait on a work item's copies in launches from now on:
// the gmi_set_wait_polls setting capped at kWaitPolls (0 gives up at once,
// which exercises the error path; negative: kWaitPolls).  The wait for copies
// still in flight after a give-up always keeps kWaitPolls.
long long wait_polls_setting();   // api.cu: the gmi_set_wait_polls setting

unsigned stage_wait_polls() {
  const long long v = wait_polls_setting();
  return v < 0 ? kWaitPolls : (unsigned)std::min<long long>(v, (long long)kWaitPolls);
}

// One warp's shared-memory area.
template <int CAP>
struct __align__(16) StageBuf {
  float4 col[CAP];                // staged colours (padded to four channels)
  float2 pos[CAP];                // staged positions
  unsigned tab[32][kPassRows + 1];  // per lane: its non-empty staged segments in walk
                                  //   order, start | end << 16 (a pad column spreads
                                  //   the lanes over the banks)
  uint2 desc[kPassRows];          // per window row: (first record, its staged index)
  uint4 item;                     // the current work item (as queued)
  unsigned act[32];               // per lane: its micro-tile takes part in the item
  unsigned long long bar;         // completes when the item's bulk copies have landed
};

template <int MTH, int MTW>
constexpr int stage_bytes() {
  return (int)sizeof(StageBuf<StageCap<MTH, MTW>::value>) * kStageWarps;
}

// Resident blocks per SM: the register budget of the accumulators (as for the
// direct-load kernel), bounded by shared memory (227 KB per SM usable).
template <int MTH, int MTW, int C>
struct StagedOcc {
  static constexpr int acc = MTH * MTW * (C + 1);
  static constexpr int regs = acc <= 32 ? 5 : (acc <= 64 ? 4 : (acc <= 80 ? 3 : 2));
  static constexpr int smem = (227 * 1024) / (stage_bytes<MTH, MTW>() + 1024);
  static constexpr int value = regs < smem ? regs : smem;
};

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arrives on the barrier and raises its expected transaction count by `bytes`.
__device__ __forceinline__ void mbar_arrive_expect(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity), "r"(kWaitHintNs)
      : "memory");
  return done != 0u;
}

// Waits for the phase of the given parity; false after `polls` polls (none:
// false at once).
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, unsigned polls = kWaitPolls) {
  for (unsigned k = 0; k < polls; ++k)
    if (mbar_test(bar, parity)) return true;
  return false;
}

// Global -> shared bulk copy on the TMA engine; `bytes` and both addresses are
// multiples of 16.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// Orders this thread's earlier shared-memory accesses before later
// async-proxy (bulk copy) writes to the same memory.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// One candidate point (position p, colour cv) into every pixel of the
// thread's micro-tile (shared sigma): separable weights gx[j] gy[r] with
// gx[j] = 2^(-(u + j sqrt(kappa))^2), u = (x_q0 - x) sqrt(kappa) (gy alike),
// then C + 1 fused multiply-adds per pixel as packed FFMA2 pairs.  Truncated
// mode keeps a pair only where -kappa d^2 >= neg_thr.
template <int MTH, int MTW, int C, bool TRUNC>
__device__ __forceinline__ void consume_pt(float2* accp, float* accs, float sk, float xq0, float yq0, float neg_thr,
                                           const float2 p, const float4 cv) {
  constexpr int NP = (C + 1) / 2;
  constexpr int ODD = (C + 1) & 1;
  const float c4[4] = {cv.x, cv.y, cv.z, cv.w};
  const float clast = c4[C - 1];   // the scalar accumulator's value (C even)
  // the coordinate difference first (its rounding is relative to the small
  // difference, not to the pixel coordinate), then the scale
  const float u = (xq0 - p.x) * sk;
  const float v = (yq0 - p.y) * sk;
  float ax[MTW], gx[MTW], ay[MTH], gy[MTH];
#pragma unroll
  for (int j = 0; j < MTW; ++j) {
    const float tt = u + (float)j * sk;
    ax[j] = -tt * tt;
    gx[j] = ex2(ax[j]);
  }
#pragma unroll
  for (int r = 0; r < MTH; ++r) {
    const float tt = v + (float)r * sk;
    ay[r] = -tt * tt;
    gy[r] = ex2(ay[r]);
  }
  if (!TRUNC) {
    // column factors times the colours once (the pair (gx, gx c_0) by one
    // scalar product), then one FFMA2 per pair and pixel
    float2 hx[MTW][NP];
    float hs[MTW];
#pragma unroll
    for (int j = 0; j < MTW; ++j) {
      hx[j][0] = make_float2(gx[j], gx[j] * c4[0]);
#pragma unroll
      for (int q = 1; q < NP; ++q) hx[j][q] = make_float2(gx[j] * c4[2 * q - 1], gx[j] * c4[2 * q]);
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
    float2 cp[NP];
    cp[0] = make_float2(1.0f, c4[0]);
#pragma unroll
    for (int q = 1; q < NP; ++q) cp[q] = make_float2(c4[2 * q - 1], c4[2 * q]);
#pragma unroll
    for (int r = 0; r < MTH; ++r)
#pragma unroll
      for (int j = 0; j < MTW; ++j) {
        const float e = ax[j] + ay[r];
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
}

// Normalises the micro-tile's sums (Eq. 1) and stores colours, den and a zero
// shift; rows of whole float4s when the micro-tile row is one.
template <int MTH, int MTW, int C>
__device__ __forceinline__ void store_tile(const ImageGeom& g, int x0, int y0, int nx, int ny, const float* acc) {
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
    if (MTW % 4 == 0 && g.vec_ok && nx == MTW) {
      float4* o = reinterpret_cast<float4*>(g.image + row * C);
#pragma unroll
      for (int k = 0; k < MTW * C / 4; ++k)
        o[k] = make_float4(outv[4 * k], outv[4 * k + 1], outv[4 * k + 2], outv[4 * k + 3]);
      if (g.den) {
        float4* dd = reinterpret_cast<float4*>(g.den + row);
#pragma unroll
        for (int k = 0; k < MTW / 4; ++k)
          dd[k] = make_float4(denv[4 * k], denv[4 * k + 1], denv[4 * k + 2], denv[4 * k + 3]);
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

// Pixels of this lane's micro-tile in warp tile wt: origin (x0, y0) and
// extent nx x ny (0 x 0 outside the image).
template <int MTH, int MTW>
__device__ __forceinline__ bool lane_tile(const ImageGeom& g, long long wt, int lane, int& x0, int& y0, int& nx,
                                          int& ny) {
  const long long lt = wt - g.wt_base;
  x0 = ((int)((unsigned)lt % (unsigned)g.wtx) * 8 + (lane & 7)) * MTW;
  y0 = ((int)((unsigned)lt / (unsigned)g.wtx) * 4 + (lane >> 3)) * MTH;
  const bool in = x0 < g.W && y0 < g.H;
  nx = in ? min(MTW, g.W - x0) : 0;
  ny = in ? min(MTH, g.H - y0) : 0;
  return in;
}

// Geometry of one work item for this thread: the warp tile's micro-tile of
// this lane, its pixels and its squared candidate radius (the plan's bound U
// plus k^2 sigma^2; +inf U marks a far-field micro-tile, left to the far kernel).
struct ItemGeo {
  long long wt;
  unsigned split, S, slot;
  int img, x0, y0, nx, ny;
  bool active;
  float R2;
};

template <int MTH, int MTW, bool TRUNC>
__device__ __forceinline__ ItemGeo item_geo(const KArgs& a, unsigned t, int lane) {
  ItemGeo it;
  uint4 item;
  float U = 0.0f;
  if ((long long)t < a.wt_total) {
    // a warp tile's first item: the tile is known before its queue entry is
    // read, so the entry and the tile's bounds are loaded together
    it.wt = t;
    item = a.w.items[t];
    if (!TRUNC) U = __ldcg(&a.w.ubound[it.wt * 32 + lane]);
  } else {
    item = a.w.items[t];
    it.wt = (long long)item.x;
    if (!TRUNC) U = __ldcg(&a.w.ubound[it.wt * 32 + lane]);
  }
  it.split = item.y & 0xffffu;
  it.S = item.y >> 16;
  it.slot = item.z;
  it.img = (int)item.w;
  const ImageGeom g = a.w.table ? a.w.table[it.img] : a.g0;   // a copy: no address of a local struct
  it.active = lane_tile<MTH, MTW>(g, it.wt, lane, it.x0, it.y0, it.nx, it.ny);
  it.R2 = g.r2k;
  if (!TRUNC) {
    if (!(U <= g.u_near_max)) it.active = false;
    it.R2 = U + g.r2k;
  }
  return it;
}

// The next work item of a warp: the queue hands out items past the first one
// of every warp; when the items do not outnumber the warps nothing is left to
// hand out, and the claim (one counter every warp would hit at about the same
// time) is skipped.
__device__ __forceinline__ unsigned claim_next(const KArgs& a, unsigned n_items, unsigned n_warps) {
  if (n_items <= n_warps) return n_items;
  return n_warps + atomicAdd(&a.w.status[kNearHead], 1u);
}

// Ring slots per lane of the pipelined direct walk (records in flight + 1;
// 8 measured no faster than 4 on the clustered batch).
constexpr int kRing = 4;

// cp.async of 8 / 16 bytes from global into shared memory (cached in L1),
// and the per-thread group commit and wait.
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Shared memory of the pipelined direct walk, in the staging buffer's records
// (which a window too large to stage leaves unused): per-lane rings of
// kRing colours and positions, laid out [slot][lane] so that lanes at the
// same step touch neighbouring words, then per lane its list of segments
// (global [start, end) pairs; rows padded by one entry against bank conflicts).
template <int CAP>
struct WalkArea {
  float4 col[kRing][32];
  float2 pos[kRing][32];
  uint2 list[32][kPassRows + 1];
};

template <int CAP>
__device__ __forceinline__ WalkArea<CAP>& walk_area(StageBuf<CAP>& sb) {
  static_assert(sizeof(WalkArea<CAP>) <= CAP * (sizeof(float4) + sizeof(float2)) + sizeof(sb.tab),
                "the walk's rings and lists fit the staging buffer's records and segment table");
  return *reinterpret_cast<WalkArea<CAP>*>(&sb.col[0]);
}

template <int CAP>
__device__ __forceinline__ uint2* walk_list(StageBuf<CAP>& sb, int lane) { return walk_area(sb).list[lane]; }

// Walks the nwalk records of the lane's nlist segments in order: the lane's
// next kRing - 1 records are always being copied into its ring slots, and
// consume(position, colour) takes each from shared memory once its copy has
// landed.  Every active lane consumes one record per step, so the slot is
// the same across the warp.
template <int CAP, typename F>
__device__ __forceinline__ void pipelined_walk(StageBuf<CAP>& sb, int lane, const float2* __restrict__ sxy,
                                               const float4* __restrict__ sval, unsigned nlist, unsigned nwalk,
                                               F&& consume) {
  WalkArea<CAP>& A = walk_area(sb);
  const uint2* L = A.list[lane];
  // producer cursor: segment kp, record ip of [ip, ep)
  unsigned kp = 0u, ip = 0u, ep = 0u;
  if (nlist > 0u) {
    const uint2 s0 = L[0];
    ip = s0.x;
    ep = s0.y;
  }
  auto issue = [&](unsigned slot) {   // the producer's next record into `slot` (if any left)
    if (kp < nlist) {
      cp_async8(&A.pos[slot][lane], &sxy[ip]);
      cp_async16(&A.col[slot][lane], &sval[ip]);
      if (++ip == ep && ++kp < nlist) {
        const uint2 sn = L[kp];
        ip = sn.x;
        ep = sn.y;
      }
    }
    cp_async_commit();   // one group per step, empty once the records run out
  };
#pragma unroll
  for (int j = 0; j < kRing - 1; ++j) issue((unsigned)j);
  for (unsigned j = 0; j < nwalk; ++j) {
    issue((j + kRing - 1) % kRing);
    cp_async_wait<kRing - 1>();   // this lane's copy for step j has landed
    const unsigned slot = j % kRing;
    consume(A.pos[slot][lane], A.col[slot][lane]);
  }
  cp_async_wait<0>();
}

template <int MTH, int MTW, int C, bool TRUNC>
__global__ void __launch_bounds__(32 * kStageWarps, StagedOcc<MTH, MTW, C>::value) near_staged_kernel(KArgs a_in) {
  constexpr int CAP = StageCap<MTH, MTW>::value;
  using Buf = StageBuf<CAP>;
  extern __shared__ __align__(16) unsigned char stage_smem[];
  const KArgs a = resolve(a_in);
  constexpr int NA = MTH * MTW * (C + 1);   // accumulators per thread
  constexpr int NP = (C + 1) / 2;           // packed accumulator pairs per pixel
  constexpr int ODD = (C + 1) & 1;          // one scalar accumulator left over (C even)
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  Buf& sb = reinterpret_cast<Buf*>(stage_smem)[warp];
  if (lane == 0) mbar_init(&sb.bar);
  __syncwarp();
  unsigned parity = 0;
  bool stalled = false;   // a bounded wait gave up (warp-uniform)

  // (the queue length is needed only past the warp tiles' first items, so
  // the first item's loads do not wait for it)
  const unsigned n_items = (unsigned)min((unsigned long long)a.wt_total + a.w.status[kItemCount],
                                         (unsigned long long)a.cap_items);
  const unsigned n_warps = gridDim.x * kStageWarps;
  unsigned t = blockIdx.x * kStageWarps + warp;
  while ((long long)t < a.wt_total || t < n_items) {
    // ---- set-up: this thread's window and share; the warp's window (when it
    // fits the buffer) staged and this thread's segment list built, else the
    // direct walk
    bool staged = false;
    unsigned nseg = 0;   // this thread's staged segments
    bool listed = false; // this thread's window rows listed for the pipelined direct walk
    unsigned nlist = 0, nwalk = 0;   // its non-empty segments and their records
    unsigned nt = 0;     // next item (lane 0), claimed early so the claim overlaps the walk
    float sk, xq0, yq0, neg_thr;
    // Accumulators in packed pairs: per pixel (r, j) the pairs (den, num_0),
    // (num_1, num_2), plus num_{C-1} alone when C is even.
    float2 accp[MTH * MTW * NP];
    float accs[MTH * MTW * ODD + 1 - ODD];
    // A warp tile's first item with a valid staging plan (single images):
    // the plan, the lane's segments and the copy ranges in one round of
    // loads, then the bulk copies.
    bool planned = false;
    if (a.w.tplan && (long long)t < a.wt_total) {
      const TilePlanRec* rec = a.w.tplan + t;
      const uint4 hdr = __ldcg(&rec->hdr);
      const unsigned lw = __ldcg(&rec->lane[lane]);
      const uint2 rc = lane < kPassRows ? __ldcg(&rec->rowc[lane]) : make_uint2(0u, 0u);
      unsigned sg[kPassRows];
#pragma unroll
      for (int k = 0; k < kPassRows; ++k) sg[k] = __ldcg(&rec->seg[k][lane]);
      if (hdr.x >> 31) {
        planned = staged = true;
        const int rows = (int)(hdr.x & 0xffffu);
        const unsigned total = hdr.y;
        const ImageGeom& g = a.g0;   // tile plans exist for single images only
        int x0, y0, nx, ny;
        lane_tile<MTH, MTW>(g, t, lane, x0, y0, nx, ny);
        sk = g.sk;
        xq0 = (float)x0 + 0.5f;
        yq0 = (float)y0 + 0.5f;
        neg_thr = -g.kappa * g.r2k;
        nseg = lw & 0xffffu;
        if (lane == 0) sb.item = make_uint4(t, 1u << 16, 0xffffffffu, 0u);
        sb.act[lane] = lw >> 31;
#pragma unroll
        for (int k = 0; k < kPassRows; ++k)
          if ((unsigned)k < nseg) sb.tab[lane][k] = sg[k];
        // every lane is past its reads of the previous item's buffer
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive_expect(&sb.bar, total * (unsigned)(sizeof(float2) + sizeof(float4)));
          nt = claim_next(a, n_items, n_warps);
        }
        __syncwarp();
        const unsigned need = rc.y & 0xffffu, abase = rc.y >> 16;
        if (lane < rows && need) {
          bulk_copy(&sb.pos[abase], a.w.sxy + rc.x, need * (unsigned)sizeof(float2), &sb.bar);
          bulk_copy(&sb.col[abase], a.w.sval + rc.x, need * (unsigned)sizeof(float4), &sb.bar);
        }
#pragma unroll
        for (int k = 0; k < MTH * MTW * NP; ++k) accp[k] = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < MTH * MTW * ODD + 1 - ODD; ++k) accs[k] = 0.0f;
        if (total > 0u) {
          const bool ok = mbar_wait(&sb.bar, parity, a.stage_wait_polls);
          if (__any_sync(full, !ok)) stalled = true;
        }
        parity ^= 1u;   // the arrival completes a phase even when nothing is copied
      }
    }
    if (!planned) {
      const ItemGeo it = item_geo<MTH, MTW, TRUNC>(a, t, lane);
      const ImageGeom g = a.w.table ? a.w.table[it.img] : a.g0;   // a copy: no address of a local struct
      // what the epilogue needs, kept in shared memory rather than live
      // through the walk
      if (lane == 0) sb.item = make_uint4((unsigned)it.wt, it.split | (it.S << 16), it.slot, (unsigned)it.img);
      sb.act[lane] = it.active ? 1u : 0u;
      sk = g.sk;
      xq0 = (float)it.x0 + 0.5f;
      yq0 = (float)it.y0 + 0.5f;
      neg_thr = -g.kappa * g.r2k;
      LaneWin w;
      int my_lo = INT_MAX, my_hi = INT_MIN;
      unsigned lo = 0u, hi = 0xffffffffu;
      float myR2 = 0.0f;
      if (it.active) {
        w = lane_window(g, it.x0, it.y0, it.nx, it.ny, it.R2);
        my_lo = w.by_lo;
        my_hi = w.by_hi;
        myR2 = it.R2;
        item_share(a, g, w, it.split, it.S, lo, hi);
      }
      const int wy_lo = warp_min(my_lo), wy_hi = warp_max(my_hi);
      const int rows = wy_hi >= wy_lo ? wy_hi - wy_lo + 1 : 0;
      bool fits = rows > 0 && rows <= kPassRows;
      if (fits) {
        // The warp's window: the warp tile's pixel rectangle (clipped to the
        // image) with the largest radius of its threads; lane r takes row r.
        // Its offsets and this thread's own rows' offsets are loaded in one
        // round trip.
        const float R2w = warp_maxf(myR2);
        const long long lt = it.wt - g.wt_base;
        const int X0 = (int)((unsigned)lt % (unsigned)g.wtx) * 8 * MTW, Y0 = (int)((unsigned)lt / (unsigned)g.wtx) * 4 * MTH;
        const LaneWin ww = lane_window(g, X0, Y0, min(8 * MTW, g.W - X0), min(4 * MTH, g.H - Y0), R2w);
        unsigned S0 = 0u, E0 = 0u;
        if (lane < rows) {
          const int by = wy_lo + lane;
          int bxw_lo, bxw_hi;
          float hxw;
          row_bins(g, ww, by, bxw_lo, bxw_hi, hxw);
          const long long rowb = g.bin_base + (long long)by * g.nbx;
          S0 = __ldg(&a.w.off[rowb + bxw_lo]);
          E0 = __ldg(&a.w.off[rowb + bxw_hi + 1]);
        }
        unsigned segs[kPassRows], sege[kPassRows];   // this thread's rows: global [start, end)
#pragma unroll
        for (int k = 0; k < kPassRows; ++k) {
          segs[k] = sege[k] = 0u;
          if (it.active && w.by_lo + k <= w.by_hi) {
            int bx_lo, bx_hi;
            float hx;
            row_bins(g, w, w.by_lo + k, bx_lo, bx_hi, hx);
            const long long rowb = g.bin_base + (long long)(w.by_lo + k) * g.nbx;
            segs[k] = __ldg(&a.w.off[rowb + bx_lo]);
            sege[k] = __ldg(&a.w.off[rowb + bx_hi + 1]);
          }
        }
        // records [S0, E0) of row r widened to even indices, so that every
        // position copy starts and ends on a 16-byte boundary
        const unsigned need = E0 > S0 ? ((E0 + 1u) & ~1u) - (S0 & ~1u) : 0u;
        unsigned incl = min(need, (unsigned)CAP + 1u);   // clamped: the sum cannot wrap
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned u = __shfl_up_sync(full, incl, o);
          if (lane >= o) incl += u;
        }
        const unsigned total = __shfl_sync(full, incl, 31);
        fits = total <= (unsigned)CAP;
        if (!fits && it.active) {
          // too many records to stage, but this thread's rows are known: its
          // share of each non-empty row segment, as global [start, end)
          // pairs in its list for the pipelined direct walk below
          uint2* L = walk_list(sb, lane);
          unsigned cum = 0;
#pragma unroll
          for (int k = 0; k < kPassRows; ++k) {
            const unsigned len = sege[k] - segs[k];
            const unsigned a0 = lo > cum ? min(lo - cum, len) : 0u;
            const unsigned b0 = hi > cum ? min(hi - cum, len) : 0u;
            cum += len;
            if (a0 < b0 && GMI_IN_BOUNDS(a.w, segs[k] + b0 - 1u, a.n_total, CK_CAND)) {
              L[nlist++] = make_uint2(segs[k] + a0, segs[k] + b0);
              nwalk += b0 - a0;
            }
          }
          listed = true;
        }
        if (fits) {
          const unsigned abase = incl - need;
          if (lane < rows) sb.desc[lane] = make_uint2(S0, abase + (S0 & 1u));
          // every lane is past its reads of the previous item's buffer
          fence_async_smem();
          __syncwarp();
          if (lane == 0) {
            mbar_arrive_expect(&sb.bar, total * (unsigned)(sizeof(float2) + sizeof(float4)));
            nt = claim_next(a, n_items, n_warps);
          }
          __syncwarp();
          if (lane < rows && need) {
            const unsigned s0 = S0 & ~1u;
            bulk_copy(&sb.pos[abase], a.w.sxy + s0, need * (unsigned)sizeof(float2), &sb.bar);
            bulk_copy(&sb.col[abase], a.w.sval + s0, need * (unsigned)sizeof(float4), &sb.bar);
          }
          if (it.active) {
            // this thread's list of non-empty segments (staged indices), with
            // its share of the sequence
            unsigned cum = 0;
#pragma unroll
            for (int k = 0; k < kPassRows; ++k) {
              if (w.by_lo + k <= w.by_hi) {
                const uint2 d = sb.desc[w.by_lo + k - wy_lo];
                const unsigned len = sege[k] - segs[k];
                const unsigned a0 = lo > cum ? min(lo - cum, len) : 0u;
                const unsigned b0 = hi > cum ? min(hi - cum, len) : 0u;
                cum += len;
                const unsigned i0 = d.y + (segs[k] - d.x) + a0, i1 = d.y + (segs[k] - d.x) + b0;
                if (i0 < i1) sb.tab[lane][nseg++] = i0 | (i1 << 16);
              }
            }
          }
          if (total > 0u) {
            const bool ok = mbar_wait(&sb.bar, parity, a.stage_wait_polls);
            if (__any_sync(full, !ok)) stalled = true;
          }
          parity ^= 1u;   // the arrival completes a phase even when nothing is copied
          staged = true;
        }
      }
#pragma unroll
      for (int k = 0; k < MTH * MTW * NP; ++k) accp[k] = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < MTH * MTW * ODD + 1 - ODD; ++k) accs[k] = 0.0f;
      if (listed) {
        // the window does not fit the buffer: this thread's segments straight
        // from global memory through a ring of records per lane in the
        // (unused) staging buffer, all but one of them in flight ahead of
        // the one consumed (cp.async; each lane waits on its own copies only)
        pipelined_walk(sb, lane, a.w.sxy, a.w.sval, nlist, nwalk, [&](const float2 p, const float4 cv) {
          consume_pt<MTH, MTW, C, TRUNC>(accp, accs, sk, xq0, yq0, neg_thr, p, cv);
        });
      } else if (!fits && it.active) {
        // more window rows than the segment list holds: straight from global
        // memory row by row (staging such windows in passes of rows that fit
        // was measured slower on dense clustered windows: each pass waits for
        // its copies)
        auto consume3 = [&](const float2 p, const float4 cv, const float4) {
          consume_pt<MTH, MTW, C, TRUNC>(accp, accs, sk, xq0, yq0, neg_thr, p, cv);
        };
        direct_walk<false>(a, g, w, lo, hi, consume3);
      }
    }
    if (stalled) break;

    // ---- the walk: this thread's records, segment after segment (a tight
    // loop over each contiguous segment; in a regular grid the lanes' segments
    // have equal lengths, so the lanes stay together)
    if (staged) {
      __syncwarp();
      const unsigned* tab = sb.tab[lane];
      for (unsigned sg = 0; sg < nseg; ++sg) {
        const unsigned te = tab[sg];
        const unsigned e = te >> 16;
        if (!GMI_IN_BOUNDS(a.w, e - 1u, CAP, CK_STAGE)) continue;
        for (unsigned i = te & 0xffffu; i < e; ++i)
          consume_pt<MTH, MTW, C, TRUNC>(accp, accs, sk, xq0, yq0, neg_thr, sb.pos[i], sb.col[i]);
      }
      __syncwarp();
    }

    // ---- epilogue: the item back from shared memory, then the split-tile
    // sums or the stores
    __syncwarp();
    ItemGeo it;
    {
      const uint4 rec = sb.item;
      it.wt = (long long)rec.x;
      it.S = rec.y >> 16;
      it.slot = rec.z;
      it.img = (int)rec.w;
    }
    const ImageGeom g = a.w.table ? a.w.table[it.img] : a.g0;   // a copy: no address of a local struct
    lane_tile<MTH, MTW>(g, it.wt, lane, it.x0, it.y0, it.nx, it.ny);
    it.active = sb.act[lane] != 0u;
    if (!staged && lane == 0) nt = claim_next(a, n_items, n_warps);

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
    if (it.S > 1 && GMI_IN_BOUNDS(a.w, it.slot, a.cap_slots, CK_SLOT)) {
      // split tile: add this item's partial sums into the tile's slot; the
      // last item to finish reads the totals and writes the pixels
      float* mine = a.w.slots + ((size_t)it.slot * 32 + lane) * NA;
      if (it.active) {
#pragma unroll
        for (int k = 0; k < NA; k += 4)
          asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(mine + k), "f"(acc[k]),
                       "f"(acc[k + 1]), "f"(acc[k + 2]), "f"(acc[k + 3])
                       : "memory");
      }
      __threadfence();
      __syncwarp();
      unsigned prev = 0;
      if (lane == 0) prev = atomicAdd(&a.w.tile_done[it.wt], 1u);
      prev = __shfl_sync(full, prev, 0);
      finish = prev == it.S - 1;
      if (finish) {
        __threadfence();
        if (it.active) {
#pragma unroll
          for (int k = 0; k < NA; k += 4) {
            const float4 q = __ldcg(reinterpret_cast<const float4*>(mine + k));
            acc[k] = q.x;
            acc[k + 1] = q.y;
            acc[k + 2] = q.z;
            acc[k + 3] = q.w;
          }
        }
      }
    }
    if (finish && it.active) store_tile<MTH, MTW, C>(g, it.x0, it.y0, it.nx, it.ny, acc);
    t = __shfl_sync(full, nt, 0);
  }
  if (stalled) {
    // report, and do not leave while this warp's bulk copies may still be
    // writing into its shared memory (the phase given up on is parity ^ 1)
    if (lane == 0) atomicOr(&a.w.status[kStatusErr], ST_TIMEOUT);
    mbar_wait(&sb.bar, parity ^ 1u);
    return;
  }
  // far-field micro-tiles queued: warps out of near work build the
  // summed-area table the far-field window search reads; with far_in_near
  // they wait until it is complete, then take the far-field micro-tiles one
  // at a time (no far kernel follows), the staging buffer holding their
  // candidate lists
  if constexpr (!TRUNC) {
    const unsigned nfar = __ldcg(&a.w.status[kFarCount]);
    if (nfar > 0u && !a.far_in_near) sat_build(a);   // for the far kernel that follows
    if (nfar > 0u && a.far_in_near) {
      static_assert(sizeof(float4) * CAP + sizeof(float2) * CAP >= sizeof(unsigned) * kFarCap,
                    "the far-field list fits the staging buffer");
      sat_build(a);
      if (!sat_wait(a)) return;
      unsigned* Lf = reinterpret_cast<unsigned*>(&sb.col[0]);
      for (;;) {
        unsigned e = 0;
        if (lane == 0) e = atomicAdd(&a.w.status[kFarHead], 1u);
        e = __shfl_sync(full, e, 0);
        if (e >= nfar || !GMI_IN_BOUNDS(a.w, e, a.mt_total, CK_FARQ_READ)) break;
        far_entry<C>(a, MTH, MTW, a.w.farq[e], Lf);
        __syncwarp();   // the list is rewritten by the next entry
      }
    }
  }
}

// Resident blocks per SM of one instantiation with its shared memory (the
// opt-in size is set on first use), cached; all devices of a process are
// taken to be alike.
template <int MTH, int MTW, int C, bool TRUNC>
static int staged_occ() {
  static const int n = [] {
    const int bytes = stage_bytes<MTH, MTW>();
    cudaFuncSetAttribute(near_staged_kernel<MTH, MTW, C, TRUNC>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, near_staged_kernel<MTH, MTW, C, TRUNC>, 32 * kStageWarps,
                                                  bytes);
    return b > 0 ? b : 1;
  }();
  return n;
}

template <int MTH, int MTW, int C>
static int staged_occ_c(bool trunc) {
  return trunc ? staged_occ<MTH, MTW, C, true>() : staged_occ<MTH, MTW, C, false>();
}

template <int MTH, int MTW>
static int staged_occ_mt(int C, bool trunc) {
  switch (C) {
    case 1: return staged_occ_c<MTH, MTW, 1>(trunc);
    case 2: return staged_occ_c<MTH, MTW, 2>(trunc);
    case 3: return staged_occ_c<MTH, MTW, 3>(trunc);
    default: return staged_occ_c<MTH, MTW, 4>(trunc);
  }
}

// Resident staged-kernel blocks per SM (each block holds kStageWarps warps).
int staged_blocks_per_sm(int mth, int mtw, int C, bool trunc) {
  const int c = C < 1 ? 1 : (C > 4 ? 4 : C);
  if (mth == 4 && mtw == 8) return staged_occ_mt<4, 8>(c, trunc);
  if (mth == 2 && mtw == 4) return staged_occ_mt<2, 4>(c, trunc);
  if (mth == 4 && mtw == 2) return staged_occ_mt<4, 2>(c, trunc);
  return staged_occ_mt<4, 4>(c, trunc);
}

template <int MTH, int MTW, int C, bool TRUNC>
static cudaError_t launch_staged_k(const KArgs& a, int grid, cudaStream_t s) {
  staged_occ<MTH, MTW, C, TRUNC>();   // sets the shared-memory opt-in once
  near_staged_kernel<MTH, MTW, C, TRUNC><<<grid, 32 * kStageWarps, stage_bytes<MTH, MTW>(), s>>>(a);
  return cudaGetLastError();
}

template <int MTH, int MTW>
static cudaError_t launch_staged_mt(const KArgs& a, bool trunc, int grid, cudaStream_t s) {
  switch (a.C) {
    case 1: return trunc ? launch_staged_k<MTH, MTW, 1, true>(a, grid, s) : launch_staged_k<MTH, MTW, 1, false>(a, grid, s);
    case 2: return trunc ? launch_staged_k<MTH, MTW, 2, true>(a, grid, s) : launch_staged_k<MTH, MTW, 2, false>(a, grid, s);
    case 3: return trunc ? launch_staged_k<MTH, MTW, 3, true>(a, grid, s) : launch_staged_k<MTH, MTW, 3, false>(a, grid, s);
    default: return trunc ? launch_staged_k<MTH, MTW, 4, true>(a, grid, s) : launch_staged_k<MTH, MTW, 4, false>(a, grid, s);
  }
}

// grid: blocks of kStageWarps warps.
cudaError_t launch_near_staged(const KArgs& a, int mth, int mtw, bool trunc, int grid, cudaStream_t s) {
  if (mth == 4 && mtw == 4) return launch_staged_mt<4, 4>(a, trunc, grid, s);
  if (mth == 4 && mtw == 8) return launch_staged_mt<4, 8>(a, trunc, grid, s);
  if (mth == 2 && mtw == 4) return launch_staged_mt<2, 4>(a, trunc, grid, s);
  if (mth == 4 && mtw == 2) return launch_staged_mt<4, 2>(a, trunc, grid, s);
  return cudaErrorInvalidValue;
}

}  // namespace gmi
