// Device-side definitions shared by the libgmi kernels (sm_103a).
//
// Problem (arXiv 2012.13257, section 2): every known point i is an isotropic
// 2D normal N(mu_i, sigma^2 I) carrying a colour c_i; pixel q of the H x W
// raster takes c(q) = sum_i c_i N(q|mu_i) / Z_q with Z_q = sum_i N(q|mu_i)
// (Eq. 1, Eq. 2); channels share the weights.  With one shared sigma the
// factor 1/(2 pi sigma^2) cancels, so the kernels work with the unnormalised
// weights 2^(-kappa d^2), kappa = log2(e) / (2 sigma^2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gmi {

constexpr int kMaxC = 4;

// Bits of the device status word (status[kStatusErr]).
enum : unsigned {
  ST_NONFINITE = 1u,   // NaN/Inf among point coordinates or values
  ST_INTERNAL = 2u,    // a consistency check failed (e.g. a list overflowed)
  ST_TIMEOUT = 4u,     // a bounded wait gave up
  ST_SIGMA = 8u,       // a per-point sigma outside its range (sigmas_ok)
  ST_BOUNDS = 16u,     // checked builds: an index failed its bounds check (the access was skipped)
  ST_CANARY = 32u,     // checked builds: a guard area after a workspace region was overwritten
  ST_BINS = 64u,       // the one-launch scan gave up at its grid barrier: the bin offsets are not valid
};

// Slots of the status/counter block at the start of every workspace.
enum : int {
  kStatusErr = 0,      // error bits
  kFarCount = 1,       // micro-tiles queued for the far-field kernel
  kNearHead = 2,       // next work item for the persistent near kernel
  kFarHead = 3,        // next far-queue entry for the far kernel
  kBwdHead = 4,        // next work item for the backward kernels
  kItemCount = 5,      // near-kernel work items past the first one of each warp tile
  kSlotCount = 6,      // partial-sum slots handed out by the plan kernel
  kFbCount = 7,        // micro-tiles queued for the backward fallback kernel
  kFbHead = 8,         // next entry of that queue
  kSigDone = 9,        // blocks of the point-centric backward that have finished
  kSatHead = 10,       // next summed-area-table column job
  kLaMax = 11,         // per-point sigmas: the largest log2 normaliser la_i (float bits; la_i >= 0)
  kBadSite = 12,       // checked builds: the first failed bounds check's site (CheckSite), 0 if none
  kBadIndex = 13,      // checked builds: its index (low 32 bits)
  kBadGuard = 14,      // checked builds: the first overwritten guard area's number + 1
  kScanArrive = 15,    // blocks of the one-launch scan past their chunk sums (its grid barrier)
  kSatDone = 16,       // summed-area-table column jobs finished
  kStatusWords = 64,
};

// True when the bin offsets of this call are not valid (the one-launch scan
// gave up at its grid barrier): every kernel that follows the offsets or the
// bin-sorted arrays leaves at once, so that nothing indexes past its arrays,
// and the call reports the timeout.  The word cannot change while those
// kernels run, so every thread takes the same decision.
__device__ __forceinline__ bool bins_invalid(const unsigned* status) {
  return (__ldcg(&status[kStatusErr]) & ST_BINS) != 0u;
}


constexpr int kPassRows = 16;     // most window bin rows the staged gather stages at once

// A warp tile's staging plan, written by the plan kernel for the staged
// gather's first work item of the tile (single-image calls):
//   hdr    (window rows | valid << 31, staged records, first window bin row, 0);
//          valid = 0: the item sets itself up (split tile, window too large)
//   rowc   per window row r: (first record copied (even), records | staged index << 16)
//   lane   per lane: non-empty segments | active << 31
//   seg    per segment k and lane: staged start | end << 16
struct TilePlanRec {
  uint4 hdr;
  uint2 rowc[kPassRows];
  unsigned lane[32];
  unsigned seg[kPassRows][32];
};

// Per-image geometry and constants, computed on the host.
struct ImageGeom {
  const float* points;   // [n,2] (x, y)
  const float* values;   // [n,C]
  float* image;          // [H,W,C]
  float* den;            // [H,W] or null
  float* shift;          // [H,W] or null
  const float* sigmas;   // per-point sigmas, pp_kind floats each (sx, sy bounded by `sigma`):
                         //   [n] sigma_i, [n,2] (sx, sy) or [n,3] (sx, sy, rho); null: every
                         //   point has `sigma`
  long long n;           // points of this image
  long long pt_base;     // first point in the concatenated point space
  long long bin_base;    // first bin in the concatenated bin space
  long long wt_base;     // first warp tile in the concatenated warp-tile space
  long long ch_base;     // first point chunk in the concatenated chunk space
  int H, W;
  int b;                 // bin edge in pixels
  int nbx, nby;          // bins across / down
  int mtx, mty;          // micro-tiles across / down
  int wtx, wty;          // warp tiles across / down (8 x 4 micro-tiles each; fewer than 2^31 per image)
  float inv_b;           // 1 / b
  float sigma;           // the shared sigma; with per-point sigmas their upper bound
  float kappa;           // log2(e) / (2 sigma^2)
  float sk;              // sqrt(kappa)
  float r2k;             // (k sigma)^2
  float u_near_max;      // largest nearest-distance bound the near kernel accepts
  float e_trunc;         // k^2 log2(e) / 2: per-point sigma keeps kappa_i d^2 <= this
  int vec_ok;            // rows of image/den/shift may use 16-byte stores
  int pp_kind;           // floats per point in sigmas: 1, 2 or 3 (0 without sigmas)
  long long px_base;     // first pixel in the concatenated pixel space
  long long mt_base;     // first micro-tile in the concatenated micro-tile space
  long long sat_base;    // first entry of this image's summed-area table ((nby+1) x (nbx+1))
  long long satj_base;   // first of its table's column jobs (32 columns each)
};

// Device pointers into a workspace.
struct DevWork {
  unsigned* status;      // [kStatusWords]
  unsigned* off;         // [nb_total + 1]: bin counts, scanned in place into offsets
  unsigned char* oob;    // [nb_total]: bin holds a point outside its image frame
  unsigned* rank;        // [n_total]: slot of each point inside its bin
  float2* sxy;           // [n_total]: bin-sorted positions
  float4* sval;          // [n_total]: bin-sorted colours, padded to 4 channels
  unsigned* partials;    // scan partial sums
  uint2* farq;           // [mt_total]: (image, micro-tile) queued for the far kernel
  uint4* items;          // [cap_items]: near-kernel work items (warp tile, split | splits << 16,
                         //   slot, image); the first item of warp tile wt is items[wt]
  unsigned* tile_done;   // [wt_total]: finished splits per warp tile
  float* slots;          // [cap_slots * slot_floats]: sums of the work items of split warp tiles
  float* ubound;         // [wt_total * 32]: per micro-tile bound U on the nearest squared
                         //   distance (+inf: far-field micro-tile), written by the plan
  unsigned* perm;        // [n_total]: input index of each bin-sorted point
  float4* spp;           // [n_total]: per-point sigma constants of each bin-sorted point
                         //   (pp_consts or pp_cov_consts); written only with sigmas
  // backward pass only
  float4* pplane;        // [pixels * (C == 4 ? 2 : 1)]: g_c / den and s' per core pixel
  unsigned* fbflag;      // [mt_total]: micro-tile holds a non-core pixel
  uint2* fbq;            // [mt_total]: queue of such micro-tiles (image, micro-tile)
  float* sig_part;       // [kSigParts]: per-block sigma-gradient partials
  float* ppmom;          // [n_total * kPpMomentFloats]: per-point moments of the exact-mode
                         //   per-point-sigma backward
  unsigned* sat;         // per image [(nby+1) x (nbx+1)]: points in bins [0,by) x [0,bx), built
                         //   by the near kernel when the far-field queue is not empty
  const ImageGeom* table;// device descriptor table (batched) or null (single image)
  TilePlanRec* tplan;    // [wt_total] staging plans of the staged gather (written by
                         //   the plan kernel), or null: the gather sets up every item itself
};

// Bounds checks of a checked build (compiled with -DGMI_CHECKED): every index
// into the workspace's queues, slots and sorted arrays that a kernel computes
// from a counter, a queue entry or another kernel's output is tested before
// the access.  A failed test skips the access, sets ST_BOUNDS and records the
// first site and index; it never traps.  Without GMI_CHECKED a check is the
// constant true and costs nothing.
enum CheckSite : unsigned {
  CK_BIN = 1,          // bin_count: the point's bin
  CK_SCATTER = 2,      // scatter: the point's slot in the sorted arrays
  CK_FARQ = 3,         // plan: far-field queue entry
  CK_STAGE = 4,        // staged gather: a segment of the staging buffer
  CK_CAND = 5,         // gathers: a candidate's sorted index
  CK_FARQ_READ = 6,    // far kernel: a queue entry read back (image, micro-tile)
  CK_FBQ = 7,          // backward: fallback queue entry
  CK_PIXEL = 8,        // backward: a pixel of the per-pixel plane
  CK_MOMENT = 9,       // per-point exact backward: a point's moments
  CK_SLOT = 10,        // split tiles: a partial-sum slot
  CK_ITEM = 11,        // near kernel: a work item index
  CK_SAT = 12,         // summed-area table entry
};

__device__ __forceinline__ bool checked_index(unsigned* status, long long i, long long n, unsigned site) {
#ifdef GMI_CHECKED
  if (i >= 0 && i < n) return true;
  atomicOr(&status[kStatusErr], ST_BOUNDS);
  if (atomicCAS(&status[kBadSite], 0u, site) == 0u) status[kBadIndex] = (unsigned)i;
  return false;
#else
  (void)status;
  (void)i;
  (void)n;
  (void)site;
  return true;
#endif
}

#define GMI_IN_BOUNDS(w, i, n, site) ::gmi::checked_index((w).status, (long long)(i), (long long)(n), (site))

struct KArgs {
  DevWork w;
  ImageGeom g0;          // the image when table == null
  int n_images;
  int C;
  long long n_total;     // points over all images
  long long nb_total;    // bins over all images
  long long wt_total;    // warp tiles over all images
  long long ch_total;    // point chunks over all images
  long long mt_total;    // micro-tiles over all images
  long long px_total;    // output pixels over all images
  long long satj_total;  // summed-area-table column jobs over all images
  unsigned cap_items;    // capacity of w.items
  unsigned cap_slots;    // capacity of w.slots, in slots
  int mth, mtw;          // micro-tile of the near kernel
  int gather;            // GMI_GATHER_* of the call (host-side choice of the near kernel)
  int far_in_near;       // the staged near kernel takes the far-field micro-tiles (no far kernel)
  unsigned stage_wait_polls;  // polls of the staged gather's first wait on its copies (gmi_set_wait_polls)
  const long long* totals;  // batched: device copy of the totals below (else null)
};

// Layout of the device totals of a batch (uploaded with its descriptor table),
// so that one captured launch sequence serves any batch within capacity.
enum : int {
  kTotImages = 0, kTotPoints, kTotBins, kTotWarpTiles, kTotChunks, kTotMicroTiles, kTotPixels, kTotSatJobs,
  kTotCount = 8
};

// Kernel arguments with the totals of a batched call read from the device.
__device__ __forceinline__ KArgs resolve(const KArgs& in) {
  KArgs a = in;
  if (in.totals) {
    a.n_images = (int)in.totals[kTotImages];
    a.n_total = in.totals[kTotPoints];
    a.nb_total = in.totals[kTotBins];
    a.wt_total = in.totals[kTotWarpTiles];
    a.ch_total = in.totals[kTotChunks];
    a.mt_total = in.totals[kTotMicroTiles];
    a.px_total = in.totals[kTotPixels];
    a.satj_total = in.totals[kTotSatJobs];
  }
  return a;
}

constexpr int kChunk = 256;             // points per chunk (one per thread) in the binning kernels
constexpr int kScanChunk = 1024;        // bins per block in the scan kernels
constexpr int kSigParts = 4096;         // sigma-gradient partials (one per backward block)
constexpr int kPpMomentFloats = 10;     // per-point moments of the exact per-point-sigma backward
constexpr int kSplitMax = 64;           // most work items one warp tile is split into
constexpr unsigned kSplitTarget = 160;  // candidates per thread per work item


// Largest image index whose base (Field 0: chunks, 1: warp tiles, 2: points,
// 3: pixels, 4: summed-area-table column jobs) is <= idx.
template <int Field>
__device__ __forceinline__ int find_image(const KArgs& a, long long idx) {
  if (a.w.table == nullptr) return 0;
  int lo = 0, hi = a.n_images - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    const ImageGeom& t = a.w.table[mid];
    const long long base = Field == 0 ? t.ch_base
                         : Field == 1 ? t.wt_base
                         : Field == 2 ? t.pt_base
                         : Field == 3 ? t.px_base
                                      : t.satj_base;
    if (base <= idx) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// 2^x on the special-function unit (flushes subnormal results to zero).
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Error-free sum (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float aa = __fsub_rn(s, bb);
  e = __fadd_rn(__fsub_rn(a, aa), __fsub_rn(b, bb));
}

// Squared distance from the pixel centre (qx, qy) to (px, py), minus a shift
// m, evaluated with error-free transformations so that the result keeps its
// absolute accuracy (~1e-7 of the result, not of d^2) when d^2 and m are both
// large and nearly equal (far-field pixels).
__device__ __forceinline__ float shifted_sqdist(float qx, float qy, float px, float py, float m) {
  float sx, ex, sy, ey;
  two_sum(qx, -px, sx, ex);
  two_sum(qy, -py, sy, ey);
  float x2 = __fmul_rn(sx, sx);
  float x2e = __fmaf_rn(sx, sx, -x2);
  float y2 = __fmul_rn(sy, sy);
  float y2e = __fmaf_rn(sy, sy, -y2);
  float t, te, u, ue;
  two_sum(x2, y2, t, te);
  two_sum(t, -m, u, ue);
  float lo = __fadd_rn(__fadd_rn(te, ue), __fadd_rn(x2e, y2e));
  lo = __fmaf_rn(2.0f * sx, ex, lo);
  lo = __fmaf_rn(2.0f * sy, ey, lo);
  return __fadd_rn(u, lo);
}

// Per-point sigma (Eq. 2 with point i's own covariance): the weight of
// point i at offset (dx, dy) is N(q | mu_i, diag(sx_i^2, sy_i^2)), which up to
// the common factor 2 pi / sigma^2 (it cancels in Eq. 1) is
//   2^(la_i - kx_i dx^2 - ky_i dy^2),  kx_i = log2(e) / (2 sx_i^2),
//   ky_i = log2(e) / (2 sy_i^2),  la_i = log2(sigma^2 / (sx_i sy_i)) >= 0,
// sigma being the bound given with the call (isotropic: sx_i = sy_i).
// Returns (sqrt(kx_i), sqrt(ky_i), la_i, 0).
__device__ __forceinline__ float4 pp_consts(float sigma, float sx, float sy) {
  constexpr float kSqrtHalfLog2e = 0.84932180028801907f;   // sqrt(log2(e) / 2)
  return make_float4(kSqrtHalfLog2e / sx, kSqrtHalfLog2e / sy, log2f(sigma / sx) + log2f(sigma / sy), 0.0f);
}

// Full covariance S_i = [[sx^2, rho sx sy], [rho sx sy, sy^2]] per point: the
// weight is N(q | mu_i, S_i), up to the same common factor
//   2^(la_i - (kxx dx^2 + kxy dx dy + kyy dy^2)),
//   kxx = log2(e) / (2 sx^2 (1 - rho^2)),  kyy = log2(e) / (2 sy^2 (1 - rho^2)),
//   kxy = -log2(e) rho / (sx sy (1 - rho^2)),
//   la_i = log2(sigma^2 / (sx sy sqrt(1 - rho^2))),
// the bracket being d^T S_i^-1 d log2(e) / 2.  Returns (kxx, kxy, kyy, la_i).
__device__ __forceinline__ float4 pp_cov_consts(float sigma, float sx, float sy, float rho) {
  constexpr float kHalfLog2e = 0.72134752044448170f;   // log2(e) / 2
  const float e = fmaf(-rho, rho, 1.0f);
  const float kxx = kHalfLog2e / (sx * sx * e), kyy = kHalfLog2e / (sy * sy * e);
  const float kxy = -2.0f * kHalfLog2e * rho / (sx * sy * e);
  return make_float4(kxx, kxy, kyy, log2f(sigma / sx) + log2f(sigma / sy) - 0.5f * log2f(e));
}

// Bin coordinate of a position along one axis, clamped to [0, nb-1]; NaN maps to 0.
__device__ __forceinline__ int bin_coord(float x, float inv_b, int nb) {
  float f = floorf(x * inv_b);
  f = fminf(fmaxf(f, 0.0f), (float)(nb - 1));   // fmaxf(NaN, 0) == 0
  return (int)f;
}

}  // namespace gmi
