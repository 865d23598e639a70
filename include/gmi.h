/*
 * gmi.h -- C ABI of libgmi: Gaussian-mixture interpolation of scattered
 * points onto an H x W raster, hand-written CUDA for sm_103a (B300).
 *
 * The operation (Skorokhodov, arXiv 2012.13257, section 2, Eq. 1 and Eq. 2):
 * every known point i is an isotropic 2D normal N(mu_i, sigma^2 I) with
 * mu_i = points[i] = (x_i, y_i) and a colour values[i] in R^C; every output
 * pixel q takes the normalised, density-weighted mean of the known colours
 *
 *     c(q) = sum_i values[i] * N(q | mu_i, sigma^2 I) / Z_q,
 *     Z_q  = sum_i N(q | mu_i, sigma^2 I),
 *
 * with the same weights for every channel (end of section 2).
 *
 * Conventions fixed by this library (the paper leaves them open):
 *   - coordinates and sigma are in output-pixel units; x runs along W
 *     (columns), y along H (rows); pixel (i, j) is queried at
 *     q = (j + 0.5, i + 0.5);
 *   - all arrays are row-major, contiguous float32: points [N,2] as (x, y),
 *     values [N,C], image [H,W,C], den/shift planes [H,W];
 *   - GMI_MODE_EXACT (default) evaluates the full sums.  A point whose
 *     squared distance exceeds m_q + k^2 sigma^2 (m_q = squared distance from
 *     q to its nearest point, k = radius_sigmas) carries less than e^{-k^2/2}
 *     of the nearest point's weight and may be skipped (k = 6: 1.5e-8);
 *   - GMI_MODE_TRUNCATED is the literal reading of the paper's "close enough"
 *     rule with radius k*sigma: only points with d <= k sigma count, and a
 *     pixel with none gets colour 0 and den 0;
 *   - N = 0 gives an all-zero image (and den 0).  Points outside the frame
 *     are allowed and contribute like any other.
 *
 * Ownership: every buffer is owned by the caller; pointers marked "device"
 * must be CUDA device (or managed) memory on the current device.  The
 * single-image and batched entry points allocate nothing: scratch memory is a
 * caller-provided workspace sized by the matching *_workspace_size call.  The
 * server owns one device pool of at most its memory budget, allocated at
 * creation.
 *
 * Asynchrony: compute calls enqueue work on `stream` and return without
 * waiting, unless params->flags has GMI_FLAG_SYNC_CHECK, in which case they
 * synchronise the stream and return the status word the kernels wrote
 * (e.g. GMI_ERR_NONFINITE for NaN/Inf inputs).  gmi_workspace_status reads
 * that word after the fact.
 *
 * Thread safety: calls on different workspaces / streams may run
 * concurrently; a workspace must not be used by two calls in flight at once.
 */
#ifndef GMI_H_
#define GMI_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t without pulling in the CUDA headers. */
typedef struct CUstream_st* gmi_stream_t;

typedef enum {
    GMI_OK = 0,
    GMI_ERR_INVALID_ARG = 1,   /* argument outside its documented range */
    GMI_ERR_NONFINITE = 2,     /* NaN/Inf in points or values (found on device) */
    GMI_ERR_WORKSPACE = 3,     /* workspace NULL, misaligned or too small */
    GMI_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    GMI_ERR_BUDGET = 5,        /* request larger than the server's memory budget */
    GMI_ERR_TIMEOUT = 6,       /* a bounded wait expired */
    GMI_ERR_UNSUPPORTED = 7,   /* valid but not built (e.g. C > 4) */
    GMI_ERR_NOT_FOUND = 8,     /* unknown server request id */
    GMI_ERR_CAPACITY = 9,      /* batch exceeds the plan's capacities */
    GMI_ERR_INTERNAL = 10      /* a device-side consistency check failed */
} gmi_status;

typedef enum { GMI_MODE_EXACT = 0, GMI_MODE_TRUNCATED = 1 } gmi_mode;

/* params->flags */
#define GMI_FLAG_SYNC_CHECK 0x1u   /* synchronise and return the device status */
/* gmi_forward and the per-point forward calls only: run the launch
 * sequence as a cached CUDA graph.  The first call with a given device, set of
 * pointers (points, values, sigmas, image, den_out, shift_out, workspace),
 * sizes (N, C, H, W, ws_bytes) and params captures it; later calls with the
 * same ones replay it (one host launch, shorter gaps between the kernels on
 * the device).  The kernels read the buffers when they run, so replay is
 * correct whatever they hold.  Up to 32 graphs are kept per process (least
 * recently used dropped).  Ignored while the stream is being captured or
 * stage profiling is on.  Worth it for repeated calls on the same buffers; a
 * call on new buffers pays one capture (~0.1-1 ms). */
#define GMI_FLAG_GRAPH 0x2u

/* Kernel variants (params->variant); 0 = choose automatically. */
#define GMI_VARIANT_AUTO 0
#define GMI_VARIANT_MT4x4 1        /* each thread owns a 4x4 pixel micro-tile */
#define GMI_VARIANT_MT4x8 2        /* 4 rows x 8 columns */
#define GMI_VARIANT_MT2x4 3        /* 2 rows x 4 columns */
#define GMI_VARIANT_MT4x2 4        /* 4 rows x 2 columns */

/* How the near-field gather reads its candidate points (params->gather).
 * Both compute the same sums; they differ only in speed. */
#define GMI_GATHER_AUTO 0          /* staged for one shared sigma, direct for per-point sigmas */
#define GMI_GATHER_STAGED 1        /* each warp stages its candidate window in shared memory
                                      (bulk copies) and its threads walk it there */
#define GMI_GATHER_DIRECT 2        /* each thread loads its candidates from global memory
                                      through the L1 cache */

typedef struct {
    float sigma;          /* std of every point's Gaussian, output px; finite, > 0 */
    float radius_sigmas;  /* k: radius rule in sigmas; finite, > 0; default 6 */
    int mode;             /* gmi_mode */
    unsigned flags;       /* GMI_FLAG_* */
    int bin_px;           /* edge of the square point bins in px; 0 = auto (1..64) */
    int variant;          /* GMI_VARIANT_*; 0 = auto */
    int gather;           /* GMI_GATHER_*; 0 = auto.  Per-point sigmas always use the
                             direct gather */
    int reserved;         /* set to 0 */
} gmi_params;

/* Library version string, e.g. "gmi 0.1.0 sm_103a". */
const char* gmi_version(void);

/* Human-readable name of a status code; never NULL. */
const char* gmi_status_string(gmi_status s);

/* Fills *p with the defaults: sigma = 1, radius_sigmas = 6, exact mode,
 * no flags, automatic bins and variant.  Returns GMI_ERR_INVALID_ARG if p is
 * NULL. */
gmi_status gmi_params_default(gmi_params* p);

/*
 * Workspace size for one gmi_forward / gmi_backward call on an N-point,
 * C-channel, H x W problem with these params.  Writes the byte count to
 * *bytes.  Errors: GMI_ERR_INVALID_ARG (N < 0, H or W < 1, sigma or k not
 * finite and > 0, bytes NULL, H*W > 2^31), GMI_ERR_UNSUPPORTED (C outside
 * 1..4).  The size does not depend on the point coordinates.
 */
gmi_status gmi_workspace_size(int64_t N, int C, int H, int W, const gmi_params* p,
                              size_t* bytes);

/*
 * Forward pass, Eq. 1 and Eq. 2 of section 2.
 *   points   device [N,2] float32 (x, y), 8-byte aligned
 *   values   device [N,C] float32
 *   image    device [H,W,C] float32, written
 *   den_out  device [H,W] float32 or NULL: the density sum scaled by the
 *            pixel's shift, sum_i exp(-(d_i^2 - shift_q)/(2 sigma^2)), over
 *            the points used (the 1/(2 pi sigma^2) factor is left out: it
 *            cancels in Eq. 1)
 *   shift_out device [H,W] float32 or NULL: the per-pixel shift used
 *            (0 where none was needed; about the nearest squared distance
 *            where the unshifted weights would underflow)
 *   workspace device, >= gmi_workspace_size bytes, 256-byte aligned; its
 *            contents on entry are ignored
 * Errors: as gmi_workspace_size, plus GMI_ERR_WORKSPACE, GMI_ERR_CUDA; with
 * GMI_FLAG_SYNC_CHECK also GMI_ERR_NONFINITE / GMI_ERR_TIMEOUT (a bounded
 * device wait gave up; see gmi_set_wait_polls) / GMI_ERR_INTERNAL.  On an
 * argument error nothing is enqueued.
 */
gmi_status gmi_forward(const float* points, const float* values, int64_t N, int C,
                       int H, int W, const gmi_params* p, float* image, float* den_out,
                       float* shift_out, void* workspace, size_t ws_bytes,
                       gmi_stream_t stream);

/*
 * Backward pass: gradients of L = sum_q sum_c grad_image[q,c] * image[q,c]
 * (the paper has forward and backward CUDA kernels but prints no backward
 * formulas; these are the chain rule on Eq. 1):
 *   grad_values[i,c] = sum_q grad[q,c] w_i(q) / Z_q
 *   grad_points[i]   = sum_q (w_i(q)/Z_q) t_i(q) (q - mu_i) / sigma^2
 *   grad_sigma       = sum_q sum_i (w_i(q)/Z_q) t_i(q) |q - mu_i|^2 / sigma^3
 *   with t_i(q) = sum_c grad[q,c] (values[i,c] - image[q,c]).
 *   image, den, shift: the outputs of the matching gmi_forward (den and shift
 *            must not be NULL); grad_image device [H,W,C]
 *   grad_points [N,2], grad_values [N,C], grad_sigma [1]: device, written
 *            (each may be NULL to skip it)
 * The point bins are rebuilt inside the call (nothing is kept from the
 * forward pass except image/den/shift).  Errors: as gmi_forward.
 */
gmi_status gmi_backward(const float* points, const float* values, int64_t N, int C,
                        int H, int W, const gmi_params* p, const float* image,
                        const float* den, const float* shift, const float* grad_image,
                        float* grad_points, float* grad_values, float* grad_sigma,
                        void* workspace, size_t ws_bytes, gmi_stream_t stream);

/*
 * Forward pass with a sigma per point: Eq. 2's normal of point i becomes
 * N(mu_i, sigmas[i]^2 I), so its normaliser 1/(2 pi sigma_i^2) no longer
 * cancels in Eq. 1 and is kept.  An extension: section 2 gives every point
 * one fixed sigma, and the point-optimisation experiment (section 3, Fig. 4)
 * finds the choice of sigma to matter more than the point positions; with
 * gmi_backward_pp a sigma per point can be fitted by gradient descent.
 * GMI_MODE_EXACT: every point counts at every pixel (Eq. 1 over all
 * points); weights are evaluated relative to the pixel's largest one, so a
 * pixel far from every point still gets its nearest points' blend, and a
 * point weighing less than exp(-k^2/2) of the largest may be left out
 * (k = radius_sigmas), as in gmi_forward's exact mode.
 * GMI_MODE_TRUNCATED: point i counts at pixel q when |q - mu_i| <= k
 * sigma_i; a pixel no point reaches gets 0.
 *   sigmas   device [N] float32, 4-byte aligned; each finite and in
 *            [p->sigma * 2^-32, p->sigma]
 *   p        p->sigma is an upper bound on every sigmas[i] (it sets the
 *            search radius, so a tight bound is faster) and the reference
 *            scale of den_out in truncated mode
 *   den_out  device [H,W] float32 or NULL.  Truncated: sum_i (sigma /
 *            sigma_i)^2 exp(-d_i^2 / (2 sigma_i^2)) over the points that
 *            count (sigma = p->sigma; with every sigma_i = sigma it is
 *            gmi_forward's den).  Exact: sum_i w_i(q) / max_j w_j(q) >= 1,
 *            w_i = exp(-d_i^2 / (2 sigma_i^2)) / sigma_i^2.  No shift plane.
 *   points, values, image, workspace (gmi_workspace_size with the same N,
 *   C, H, W and params), GMI_FLAG_GRAPH: as gmi_forward
 * Errors: as gmi_forward, plus
 * GMI_ERR_INVALID_ARG (sigmas NULL or misaligned with N > 0; with
 * GMI_FLAG_SYNC_CHECK also a sigma outside its range, found on the device,
 * and GMI_ERR_NONFINITE for a NaN/Inf sigma).  Out-of-range sigmas without
 * the check give a wrong image, never a fault.
 */
gmi_status gmi_forward_pp(const float* points, const float* values, const float* sigmas,
                          int64_t N, int C, int H, int W, const gmi_params* p,
                          float* image, float* den_out, void* workspace, size_t ws_bytes,
                          gmi_stream_t stream);

/*
 * Backward pass of gmi_forward_pp: gradients of L = sum_q sum_c
 * grad_image[q,c] image[q,c] with w_i(q) the kept weight of point i:
 *   grad_values[i,c] = sum_q grad[q,c] w_i(q) / Z_q
 *   grad_points[i]   = sum_q (w_i(q)/Z_q) t_i(q) (q - mu_i) / sigma_i^2
 *   grad_sigmas[i]   = sum_q (w_i(q)/Z_q) t_i(q) (|q - mu_i|^2 / sigma_i^3
 *                      - 2 / sigma_i)
 *   with t_i(q) as for gmi_backward.  image, den: the outputs of the matching
 *   gmi_forward_pp (den must not be NULL; exact mode recomputes each pixel's
 *   sums and reads neither); grad_points [N,2], grad_values [N,C],
 *   grad_sigmas [N]: device, written (each may be NULL to skip it).
 * Truncated mode writes each gradient from one thread (no atomics): the
 * result does not vary from run to run.  Exact mode adds every (pixel,
 * point) term into per-point sums with float atomics, so its low bits can
 * vary between runs.  Errors: as gmi_forward_pp.
 */
gmi_status gmi_backward_pp(const float* points, const float* values, const float* sigmas,
                           int64_t N, int C, int H, int W, const gmi_params* p,
                           const float* image, const float* den, const float* grad_image,
                           float* grad_points, float* grad_values, float* grad_sigmas,
                           void* workspace, size_t ws_bytes, gmi_stream_t stream);

/*
 * Forward and backward passes with an axis-aligned covariance per point:
 * point i is N(mu_i, diag(sx_i^2, sy_i^2)) with its normaliser
 * 1/(2 pi sx_i sy_i) kept; in truncated mode it counts at pixel q inside
 * its ellipse dx^2/sx_i^2 + dy^2/sy_i^2 <= k^2, in exact mode everywhere
 * (relative to the pixel's largest weight, as gmi_forward_pp).  With sx_i = sy_i
 * they compute what gmi_forward_pp / gmi_backward_pp compute.
 *   sigmas_xy      device [N,2] float32 (sx, sy) per point, 4-byte aligned;
 *                  each finite and in [p->sigma * 2^-32, p->sigma]
 *   den_out / den  truncated: sum_i sigma^2 / (sx_i sy_i) exp(-(dx^2/sx_i^2
 *                  + dy^2/sy_i^2) / 2) over the points that count; exact:
 *                  the weights' sum relative to the largest (as
 *                  gmi_forward_pp)
 *   grad_points    [N,2]: sum_q (w_i/Z_q) t_i(q) (dx / sx_i^2, dy / sy_i^2)
 *   grad_sigmas_xy [N,2]: sum_q (w_i/Z_q) t_i(q) (dx^2/sx_i^3 - 1/sx_i,
 *                  dy^2/sy_i^3 - 1/sy_i)
 * Everything else (arguments, workspace, flags, errors, determinism of the
 * backward) as for gmi_forward_pp / gmi_backward_pp.
 */
gmi_status gmi_forward_aniso(const float* points, const float* values, const float* sigmas_xy,
                             int64_t N, int C, int H, int W, const gmi_params* p,
                             float* image, float* den_out, void* workspace, size_t ws_bytes,
                             gmi_stream_t stream);

gmi_status gmi_backward_aniso(const float* points, const float* values, const float* sigmas_xy,
                              int64_t N, int C, int H, int W, const gmi_params* p,
                              const float* image, const float* den, const float* grad_image,
                              float* grad_points, float* grad_values, float* grad_sigmas_xy,
                              void* workspace, size_t ws_bytes, gmi_stream_t stream);

/*
 * Forward and backward passes with a full covariance per point: point i is
 * N(mu_i, S_i), S_i = [[sx^2, rho sx sy], [rho sx sy, sy^2]], with its
 * normaliser 1/(2 pi sqrt(det S_i)) kept; in truncated mode it counts at
 * pixel q inside its rotated ellipse d^T S_i^-1 d <= k^2, in exact mode
 * everywhere (as gmi_forward_pp).  With rho = 0
 * they compute what gmi_forward_aniso / gmi_backward_aniso compute.  The cross
 * term of the quadratic form does not factorise into a column and a row
 * factor, so every (pixel, candidate) takes its own exponential.
 *   cov         device [N,3] float32 (sx, sy, rho) per point, 4-byte aligned;
 *               finite, sx, sy >= p->sigma * 2^-32, |rho| <= 0.99 (nearer 1
 *               the quadratic form's terms grow as 1/(1 - rho^2) and float32
 *               loses the accuracy the forward promises)
 *   p           p->sigma bounds the square root of the largest eigenvalue of
 *               every S_i (a rotated ellipse reaches k sqrt(lambda_max) from
 *               its centre, which can exceed k max(sx, sy)); checked on the
 *               device to a relative 2^-20
 *   den_out/den truncated: sum_i sigma^2 / sqrt(det S_i) exp(-d^T S_i^-1
 *               d / 2) over the points that count; exact: relative to the
 *               largest weight (as gmi_forward_pp)
 *   grad_points [N,2]: sum_q (w_i/Z_q) t_i(q) S_i^-1 d
 *   grad_cov    [N,3]: d/d(sx, sy, rho) of L, from the chain rule on
 *               ln w_i = -d^T S_i^-1 d / 2 - ln sx - ln sy - ln(1 - rho^2) / 2
 * Everything else as for gmi_forward_pp / gmi_backward_pp.
 */
gmi_status gmi_forward_cov(const float* points, const float* values, const float* cov,
                           int64_t N, int C, int H, int W, const gmi_params* p,
                           float* image, float* den_out, void* workspace, size_t ws_bytes,
                           gmi_stream_t stream);

gmi_status gmi_backward_cov(const float* points, const float* values, const float* cov,
                            int64_t N, int C, int H, int W, const gmi_params* p,
                            const float* image, const float* den, const float* grad_image,
                            float* grad_points, float* grad_values, float* grad_cov,
                            void* workspace, size_t ws_bytes, gmi_stream_t stream);

/*
 * Where gmi_forward leaves the binned points in its workspace (byte offsets
 * from the workspace start), for inspection and tests of the binning step
 * (section 2's "close enough" points, found through bins of b x b pixels):
 *   off  [nbx*nby + 1] uint32: exclusive prefix sums of the bin counts
 *        (off[nb] = N); bin = by * nbx + bx, bx = clamp(floor(x / b), 0,
 *        nbx - 1), by likewise from y;
 *   oob  [nbx*nby] uint8: 1 where the bin holds a point outside [0,W)x[0,H);
 *   sxy  [N] float2, sval [N] float4 (colours padded with 0), perm [N]
 *        uint32: the points sorted by bin (sxy[k] = points[perm[k]]); the
 *        order inside a bin is unspecified;
 *   ubound [wtx*wty*32] float, exact mode: per micro-tile of mth x mtw pixels
 *        an upper bound U on the squared distance from each of its pixels to
 *        the nearest point (+inf: the micro-tile went to the far-field
 *        kernel); entry (wt * 32 + l) is micro-tile (l % 8, l / 8) of warp
 *        tile wt = wty_index * wtx + wtx_index (8 x 4 micro-tiles each);
 *   sat  [(nby+1)*(nbx+1)] uint32, exact mode, built only when the plan sent
 *        micro-tiles to the far-field kernel: entry (by, bx) = points in
 *        bins [0, by) x [0, bx) (row stride nbx + 1).
 * Valid after a gmi_forward call with N > 0 on that workspace has finished.
 * Errors: GMI_ERR_INVALID_ARG (as gmi_workspace_size).
 */
typedef struct {
    size_t off, oob, sxy, sval, perm;  /* byte offsets into the workspace */
    int bin_px, nbx, nby;               /* bin edge in pixels, bins across and down */
    size_t total;                       /* gmi_workspace_size */
    size_t ubound;                      /* byte offset of the micro-tile bounds */
    int mth, mtw, wtx, wty;             /* micro-tile rows x columns; warp tiles across, down */
    size_t sat;                         /* byte offset of the summed-area table */
} gmi_ws_layout;

gmi_status gmi_workspace_layout(int64_t N, int C, int H, int W, const gmi_params* p,
                                gmi_ws_layout* out);

/*
 * Reads the device status word of a workspace after its stream has finished
 * (synchronises `stream` first).  Returns GMI_OK, GMI_ERR_NONFINITE,
 * GMI_ERR_INVALID_ARG (a per-point sigma out of range), GMI_ERR_TIMEOUT (a
 * bounded device wait gave up) or GMI_ERR_INTERNAL for the last call that
 * used the workspace.
 */
gmi_status gmi_workspace_status(const void* workspace, gmi_stream_t stream);

/*
 * Memory-safety checks of a checked build (no counterpart in the paper; the
 * library built with -DGMI_CHECKED, libgmi_checked.so, stands in for a
 * sanitizer).  Such a build tests every index it derives from a counter, a
 * queue entry or another kernel's output before using it (a failed test
 * skips the access and records where), and leaves a 256-byte guard area
 * after every workspace region, written with a known pattern at the start of
 * each call.  Its workspaces are larger: size them with this build's
 * gmi_workspace_size.  Other builds return GMI_ERR_UNSUPPORTED from both calls
 * and 0 from gmi_is_checked_build.
 *
 * gmi_check_workspace: after a single-image call (forward, backward, per
 * point) with the same N, C, H, W and params on `workspace` (ws_bytes as
 * given to that call), tests the guard areas on `stream`, synchronises it
 * and returns GMI_OK when no bounds check failed and every guard is intact,
 * else GMI_ERR_INTERNAL.  report (NULL or uint32_t[4]): the status bits, the
 * first failed check's site (CheckSite in the sources) and index, the first
 * overwritten guard's number + 1.
 * gmi_batch_check_workspace: the same for a batched plan's workspace after
 * a batched call.
 */
struct gmi_batch_plan;   /* opaque, see gmi_batch_plan_create */
gmi_status gmi_check_workspace(int64_t N, int C, int H, int W, const gmi_params* p,
                               void* workspace, size_t ws_bytes, gmi_stream_t stream,
                               uint32_t* report);
gmi_status gmi_batch_check_workspace(const struct gmi_batch_plan* plan, gmi_stream_t stream,
                                     uint32_t* report);
int gmi_is_checked_build(void);

/*
 * Autotuner core (the batching pattern's choice of micro-tile and bin edge;
 * no counterpart in the paper): times gmi_forward on the caller's problem for
 * every micro-tile variant (GMI_VARIANT_MT4x4, MT4x8, MT2x4) and every bin
 * edge bins[0..n_bins) (0 = the automatic rule), one warm-up and `reps` timed
 * runs each, with CUDA events on `stream`; writes *p with the fastest variant
 * and bin_px into *best, and, when times_ms is not NULL, the median time per
 * candidate into times_ms[variant_index * n_bins + bin_index] (variant order
 * as listed).  points/values as for gmi_forward.  A tuning call, not the hot
 * path: it allocates (and frees) its own workspace and output, and returns
 * after the last run (synchronous).
 * Errors: GMI_ERR_INVALID_ARG (p, bins or best NULL, n_bins < 1, reps < 1, a
 * bin edge outside [0, 1024]), the errors of gmi_workspace_size and
 * gmi_forward, GMI_ERR_CUDA.
 */
gmi_status gmi_autotune(const float* points, const float* values, int64_t N, int C, int H, int W,
                        const gmi_params* p, const int* bins, int n_bins, int reps, gmi_params* best,
                        float* times_ms, gmi_stream_t stream);

/*
 * Forward pass without a caller-provided workspace (the paper has no
 * counterpart: this is an integration convenience).
 *
 * Some callers cannot allocate device memory at all: plug-ins running inside
 * a host application that owns the GPU memory pool, latency-critical loops in
 * which a cudaMalloc/cudaFree would stall the device, and bindings whose own
 * API has no way to size and pass a workspace.  This entry point takes the
 * same arguments as gmi_forward minus the workspace and computes the same
 * result, using as scratch one statically sized device array of
 * GMI_NOALLOC_SCRATCH_BYTES that lives in the library (every GPU that loads
 * the library holds it until the process exits).  It calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *
 *   - Limit: the forward uses only the leading part of the workspace layout
 *     (gmi_workspace_size less the backward pass's planes); problems whose
 *     forward part exceeds GMI_NOALLOC_SCRATCH_BYTES are rejected with
 *     GMI_ERR_CAPACITY before anything is enqueued.  A 768x768 output from
 *     147,456 points with C = 3 needs about 21 MiB and fits; a 1024x1024
 *     output from 262,144 points needs about 37 MiB and does not: use
 *     gmi_forward beyond the limit.
 *   - Every call looks up the device address of the array on the current
 *     device (cudaGetSymbolAddress, which allocates nothing); the first call
 *     on a device loads the library's device code there, so make that first
 *     call before any stream capture.
 *   - Every call on a device shares the one array, which keeps the previous
 *     call's contents (the call clears what must start at zero itself).
 *     Calls that overlap on the GPU race on it: serialise them, e.g. issue
 *     them on one stream.
 * Errors: as gmi_forward, plus GMI_ERR_CAPACITY.
 */
#define GMI_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)

gmi_status gmi_forward_noalloc(const float* points, const float* values, int64_t N, int C,
                               int H, int W, const gmi_params* p, float* image,
                               float* den_out, float* shift_out, gmi_stream_t stream);

/* ------------------------------------------------------------------------
 * The forward pass end to end from HOST memory (the problem statement's call,
 * section 2 / Eq. 1, with the transfers included): uploads points [N,2] and
 * values [N,C] from host buffers, runs gmi_forward's pipeline on device
 * copies, and downloads the image [H,W,C] into a host buffer, all in order
 * on `stream`.  Asynchronous: image_host holds the result once the stream
 * has passed the call (synchronise before reading it).  Host buffers should
 * be pinned (cudaHostAlloc / cudaHostRegister); pageable ones work, with
 * copies the driver stages synchronously, and are never captured in a graph.
 *
 * workspace: device memory, 256-byte aligned, of at least
 * gmi_forward_host_workspace_size() bytes; it holds the forward's workspace
 * and the device copies of points, values and image.  Flags as gmi_forward;
 * with GMI_FLAG_GRAPH and pinned buffers the two uploads, the kernels and the
 * download replay as one cached CUDA graph for the same buffers and sizes.
 * No den or shift planes (use gmi_forward for those).
 * Errors: as gmi_forward.
 * ---------------------------------------------------------------------- */
gmi_status gmi_forward_host_workspace_size(int64_t N, int C, int H, int W, const gmi_params* p,
                                           size_t* bytes);
gmi_status gmi_forward_host(const float* points_host, const float* values_host, int64_t N, int C,
                            int H, int W, const gmi_params* p, float* image_host, void* workspace,
                            size_t ws_bytes, gmi_stream_t stream);

/* ------------------------------------------------------------------------
 * Measurement aid (no counterpart in the paper): while enabled, the compute
 * entry points bracket each stage of their pipeline with CUDA events recorded
 * on their own stream, so kernel times can be read without a profiler.
 * ---------------------------------------------------------------------- */
typedef enum {
    GMI_STAGE_BIN = 0,       /* memset + count + scan + scatter + plan */
    GMI_STAGE_NEAR = 1,      /* near-field gather */
    GMI_STAGE_FAR = 2,       /* far-field gather */
    GMI_STAGE_BACKWARD = 3,  /* backward gathers (after re-binning) */
    GMI_STAGE_COUNT = 4
} gmi_stage;

/* Turns stage timing on (creates a pool of CUDA events on first use) or off.
 * Process-wide.  Errors: GMI_ERR_CUDA. */
gmi_status gmi_profile_enable(int on);

/* Waits for every recorded stage, adds the elapsed milliseconds per stage
 * into ms[GMI_STAGE_COUNT] and the number of timed launches into
 * launches[GMI_STAGE_COUNT] (either may be NULL), and with reset != 0 forgets
 * them.  Stages recorded while the event pool was exhausted are not counted. */
gmi_status gmi_profile_read(double* ms, int* launches, int reset);

/* Measurement aid (no counterpart in the paper): the issue rates of the units
 * the near-field gather is bound by, measured on the current device with
 * streams of independent dependency chains, one 1024-thread block per SM
 * timed by the SM's own clock.  Writes, per SM per clock,
 *   rates[0]  ex2.approx.ftz.f32 results (the SFU),
 *   rates[1]  FP32 fused multiply-adds issued as FFMA,
 *   rates[2]  FP32 fused multiply-adds issued as packed FFMA2 (two each).
 * Synchronous (device-wide), a few milliseconds; allocates and frees two small
 * device buffers.  Errors: GMI_ERR_INVALID_ARG (rates NULL), GMI_ERR_CUDA. */
gmi_status gmi_measure_unit_rates(double* rates);

/* Test aid for the device-side bounded waits (no counterpart in the paper).
 * Two waits can give up without harm, and each records a timeout in the
 * workspace's status word, so that a GMI_FLAG_SYNC_CHECK call returns
 * GMI_ERR_TIMEOUT and the context stays usable:
 *   - the one-launch bin-count scan of single images waits at a grid
 *     barrier (at most 2^20 polls, about 0.1 s); a block that gives up also
 *     marks the bin offsets invalid, and the kernels after it then keep to
 *     their arrays and do no gather work;
 *   - the near-field gather's staged path waits on an mbarrier for each work
 *     item's bulk copies (at most 10,000 polls, about a second); a warp that
 *     gives up waits (with the full limit) for its copies still in flight
 *     and leaves.
 * This sets, process-wide, how many polls those waits get in launches made
 * from now on: polls >= 0 (0: give up at once; each wait keeps at most its
 * own default), negative: back to the defaults.  CUDA graphs captured
 * earlier keep the values they were captured with.  Always GMI_OK. */
gmi_status gmi_set_wait_polls(int64_t polls);

/* ------------------------------------------------------------------------
 * Batched forward: B independent images of uneven size in one persistent
 * launch over a global tile queue (the shapes live in a device descriptor
 * table, so one captured CUDA graph replays for any batch within capacity).
 * ---------------------------------------------------------------------- */
typedef struct {
    const float* points;   /* device [N,2] */
    const float* values;   /* device [N,C] */
    float* image;          /* device [H,W,C] */
    float* den;            /* device [H,W] or NULL */
    float* shift;          /* device [H,W] or NULL */
    int64_t N;             /* >= 0 */
    int H, W;              /* >= 1 */
    float sigma;           /* finite, > 0 */
    int bin_px;            /* 0 = auto */
} gmi_image_desc;

typedef struct gmi_batch_plan gmi_batch_plan;   /* opaque */

/*
 * Creates a batch plan for up to max_images images holding at most
 * max_points points and max_pixels output pixels in total, C channels.
 * Allocates its device workspace and pinned host staging once (setup, not
 * hot path).  params supplies k, mode and the variant; its sigma is unused
 * (each image has its own).  Errors: GMI_ERR_INVALID_ARG,
 * GMI_ERR_UNSUPPORTED, GMI_ERR_CUDA (allocation failed).
 */
gmi_status gmi_batch_plan_create(int max_images, int64_t max_points, int64_t max_pixels,
                                 int C, const gmi_params* params, gmi_batch_plan** plan);

/* Frees a plan (synchronises its last launch first).  NULL is a no-op. */
gmi_status gmi_batch_plan_destroy(gmi_batch_plan* plan);

/* Device bytes the plan holds. */
size_t gmi_batch_plan_bytes(const gmi_batch_plan* plan);

/*
 * Runs the forward pass of B images (descs is a host array) in one batched
 * pipeline on `stream`: one segmented binning pass, then one persistent
 * gather over the work queue of all images' tiles.  With use_graph != 0 the
 * kernel sequence is captured into a CUDA graph on the first call and
 * replayed afterwards.  Two staging slots alternate: a call waits (host
 * side) only for the forward two calls back, whose slot it reuses.  The calls
 * on one plan share its workspace and must be ordered on one stream.
 * Errors: GMI_ERR_INVALID_ARG, GMI_ERR_CAPACITY,
 * GMI_ERR_CUDA; with GMI_FLAG_SYNC_CHECK in the plan's params, also the
 * device status.
 */
gmi_status gmi_forward_batched(gmi_batch_plan* plan, const gmi_image_desc* descs, int B,
                               int use_graph, gmi_stream_t stream);

/* Per-image arguments of the batched backward pass (see gmi_backward). */
typedef struct {
    const float* points;     /* device [N,2], as in the forward */
    const float* values;     /* device [N,C] */
    const float* image;      /* device [H,W,C]: forward output */
    const float* den;        /* device [H,W]: forward den (not NULL) */
    const float* shift;      /* device [H,W]: forward shift (not NULL) */
    const float* grad_image; /* device [H,W,C]: upstream gradient */
    float* grad_points;      /* device [N,2] or NULL */
    float* grad_values;      /* device [N,C] or NULL */
    float* grad_sigma;       /* device [1] or NULL */
    int64_t N;
    int H, W;
    float sigma;
    int bin_px;              /* 0 = auto; use the value the forward used */
} gmi_grad_desc;

/*
 * Backward pass of B images (descs is a host array) in one batched pipeline
 * on `stream`: one segmented re-binning, then the per-pixel preparation, the
 * point-centric gradient kernel and the fallback kernel over all images at
 * once (gradients as in gmi_backward).  Uses the plan's workspace, so the
 * calls on one plan (forward and backward) must be ordered on one stream; a
 * call returns once its descriptor tables are staged (two pinned staging
 * buffers alternate, so the host may prepare the next call while the previous
 * one runs).  The sigma gradients are accumulated with float atomics, so
 * their last bits may differ between runs.
 * Errors: GMI_ERR_INVALID_ARG, GMI_ERR_CAPACITY, GMI_ERR_CUDA.
 */
gmi_status gmi_backward_batched(gmi_batch_plan* plan, const gmi_grad_desc* descs, int B,
                                gmi_stream_t stream);

/*
 * Equal-shaped batches given as stacked arrays: image i of B has N points
 * at points + i*N*2 and values + i*N*C, its output at image + i*H*W*C and
 * den/shift + i*H*W, its sigma sigmas[i] (a HOST array of B floats); the
 * gradients likewise (grad_sigma + i).  The same as gmi_forward_batched /
 * gmi_backward_batched with the descriptors built from these strides, which
 * saves a caller holding [B, ...] tensors from building B descriptors.
 * den, shift may be NULL in the forward; in the backward they and image,
 * grad_image must not be.  Errors: as the batched calls, and
 * GMI_ERR_INVALID_ARG for B outside [1, the plan's max_images] or a NULL
 * sigmas.
 */
gmi_status gmi_forward_stacked(gmi_batch_plan* plan, const float* points, const float* values,
                               int B, int64_t N, int H, int W, const float* sigmas,
                               float* image, float* den, float* shift, int use_graph,
                               gmi_stream_t stream);

gmi_status gmi_backward_stacked(gmi_batch_plan* plan, const float* points, const float* values,
                                int B, int64_t N, int H, int W, const float* sigmas,
                                const float* image, const float* den, const float* shift,
                                const float* grad_image, float* grad_points, float* grad_values,
                                float* grad_sigma, gmi_stream_t stream);

/* ------------------------------------------------------------------------
 * Serving: a persistent request loop with continuous batching.  Requests are
 * admitted while their device memory fits the budget, their points are binned
 * and kept on the device, admitted requests are packed into batched launches,
 * and each request completes on its own event.
 * ---------------------------------------------------------------------- */
typedef struct gmi_server gmi_server;   /* opaque */

typedef struct {
    size_t budget_bytes;     /* device memory the server may hold in total */
    int max_batch_images;    /* images per batched launch (>= 1) */
    int64_t max_batch_pixels;/* output pixels per batched launch (>= 1) */
    int n_streams;           /* launches that may be in flight at once (1..8) */
    int C;                   /* channels (1..4) */
    float radius_sigmas;     /* k, default 6 */
    int mode;                /* gmi_mode */
    int reserved;
} gmi_server_config;

/* Fills a config with defaults (40 GB budget, 64 images, 2^25 pixels per
 * batch, 2 streams, C = 3, k = 6, exact mode). */
gmi_status gmi_server_config_default(gmi_server_config* cfg);

/* Creates the server: allocates its device pool (budget_bytes) and starts
 * its launcher and completion threads.  Errors: GMI_ERR_INVALID_ARG,
 * GMI_ERR_CUDA. */
gmi_status gmi_server_create(const gmi_server_config* cfg, gmi_server** out);

/*
 * Submits one request.  points/values/image are HOST buffers (pinned memory
 * gives asynchronous copies); they must stay valid until the request
 * completes.  The request is queued until its device footprint fits the
 * budget.  *id receives the request id.  Errors: GMI_ERR_INVALID_ARG,
 * GMI_ERR_BUDGET (the request alone exceeds the budget).
 */
gmi_status gmi_server_submit(gmi_server* s, const float* points, const float* values,
                             int64_t N, int H, int W, float sigma, float* image,
                             uint64_t* id);

/*
 * Waits up to timeout_ms (< 0: forever) for request `id`.  Returns GMI_OK
 * when its image is in the host buffer, GMI_ERR_TIMEOUT, GMI_ERR_NOT_FOUND,
 * or the request's own error.  On success *latency_s (if not NULL) holds
 * the time from submission to completion, in seconds.
 */
gmi_status gmi_server_wait(gmi_server* s, uint64_t id, int timeout_ms, double* latency_s);

/* Non-blocking: GMI_OK if done, GMI_ERR_TIMEOUT if still pending. */
gmi_status gmi_server_poll(gmi_server* s, uint64_t id);

/*
 * Submits one request whose buffers are DEVICE memory on the server's device
 * (points [N,2] 8-byte aligned, values [N,C], image [H,W,C]).  Nothing is
 * copied: the batched forward reads the inputs and writes the image in place,
 * so the request takes none of the server's pool.  The buffers must stay
 * valid, and the inputs unchanged, until the request completes.  Errors: as
 * gmi_server_submit, and GMI_ERR_INVALID_ARG when a buffer is not device
 * memory of the server's device.
 */
gmi_status gmi_server_submit_device(gmi_server* s, const float* points, const float* values,
                                    int64_t N, int H, int W, float sigma, float* image,
                                    uint64_t* id);

/* Server counters: completed requests, batched launches, pixels served, and
 * the device bytes currently held by admitted requests. */
gmi_status gmi_server_stats(gmi_server* s, uint64_t* completed, uint64_t* launches,
                            uint64_t* pixels, size_t* bytes_in_use);

typedef struct {
    uint64_t completed;      /* requests completed */
    uint64_t launches;       /* batched launches queued */
    uint64_t pixels;         /* output pixels served */
    size_t bytes_in_use;     /* pool bytes held by admitted requests */
    int in_flight;           /* batches queued on the GPU and not yet seen complete */
    int max_in_flight;       /* the most that were at any one time */
    uint64_t reserved[4];
} gmi_server_counters;

/* All counters at once (the in-flight figures show whether batches overlapped
 * on the device). */
gmi_status gmi_server_get_counters(gmi_server* s, gmi_server_counters* out);

/*
 * Per-request log: from now on every completed request appends one JSON line
 * to the file at `path` (truncated first): id, device (1 for device buffers),
 * N, H, W, batch (launch number), slot (stream slot), status, and the times in
 * seconds since the server was created at which it was submitted, admitted
 * (pool memory reserved and taken into a batch), launched (its batch queued on
 * the GPU) and done (its batch's completion seen by the server, within ~20 us).
 * NULL closes the log.  Errors: GMI_ERR_INVALID_ARG if the file cannot be
 * opened.
 */
gmi_status gmi_server_set_log(gmi_server* s, const char* path);

/* Drains pending requests, stops the threads and frees the pool. */
gmi_status gmi_server_destroy(gmi_server* s);

#ifdef __cplusplus
}
#endif

#endif /* GMI_H_ */
