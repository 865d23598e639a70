/*
 * FP64 brute-force oracle for Gaussian-mixture interpolation on a
 * non-uniform grid (Skorokhodov, "Interpolating Points on a Non-Uniform
 * Grid using a Mixture of Gaussians", arXiv 2012.13257).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; it is used by the tests, by the smoke check and by the
 * benchmark's CPU-baseline leg.  It shares no code with the CUDA library.
 *
 * What is computed (paper section 2):
 *   Every known point i is an isotropic 2D normal N(mu_i, sigma^2 I) with
 *   mu_i = (x_i, y_i) and a colour c_i in R^C (section 1 introduces
 *   f: p -> c; section 2 fixes the diagonal covariance sigma^2 I with one
 *   shared sigma).  The colour at a query pixel q is the expectation
 *       c(q) = sum_i c_i N(q | mu_i, sigma^2 I) / Z_q            (Eq. 1)
 *       Z_q  = sum_i N(q | mu_i, sigma^2 I)                       (Eq. 2)
 *   and every channel is interpolated independently with the same weights
 *   (end of section 2).
 *
 * Readings of what the paper leaves open:
 *   - Query grid: the H x W output raster (section 1); pixel (i, j) (row i,
 *     column j) is queried at q = (j + 0.5, i + 0.5) in output-pixel units;
 *     x runs along W, y along H.
 *   - EXACT mode (default): the full sums of Eq. 1 and Eq. 2.  Because sigma
 *     is shared, the Gaussian normaliser 1/(2 pi sigma^2) cancels in the
 *     ratio, and so does any common factor exp(m/(2 sigma^2)); with
 *     m = min_i |q - mu_i|^2 the evaluation below is Eq. 1 written with
 *     weights w_i = exp(-(d_i^2 - m)/(2 sigma^2)) in [0, 1], which cannot
 *     underflow to 0/0 (the unshifted weights do, even in FP64, once
 *     d^2/(2 sigma^2) > ~745).
 *   - TRUNCATED mode: the paper says only points "close enough" to the query
 *     are considered but gives no radius.  This mode is the literal reading
 *     with radius k*sigma: sums over d_i <= k sigma of the unshifted weights
 *     exp(-d_i^2/(2 sigma^2)); a pixel with no point inside the disc gets
 *     colour 0 and Z = 0.
 *   - N = 0: colour 0 and Z = 0 everywhere.
 *   - Backward (the paper has CUDA forward and backward kernels but prints no
 *     formulas; the derivation is the chain rule applied to Eq. 1):
 *       dc_c(q)/dc_{i,c}  = w_i / Z
 *       dc_c(q)/dmu_i     = (w_i / Z) (c_{i,c} - c_c(q)) (q - mu_i) / sigma^2
 *       dc_c(q)/dsigma    = sum_i (w_i / Z) (c_{i,c} - c_c(q)) d_i^2 / sigma^3
 *     The shift m and the truncation boundary carry no derivative (the shift
 *     cancels exactly; the boundary is a measure-zero set).
 *
 * All arithmetic is double precision on the float32 inputs; exp() is libm.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_EXACT 0
#define ORACLE_TRUNCATED 1

/* Pixel index -> query position (section 1: the output is an H x W raster;
 * the pixel-centre convention is this oracle's reading). */
static void pixel_centre(int64_t p, int64_t W, double* qx, double* qy) {
    int64_t i = p / W, j = p % W;
    *qx = (double)j + 0.5;
    *qy = (double)i + 0.5;
}

static double sqdist(const float* points, int64_t i, double qx, double qy) {
    double dx = qx - (double)points[2 * i];
    double dy = qy - (double)points[2 * i + 1];
    return dx * dx + dy * dy;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Forward pass, Eq. 1 and Eq. 2, at a list of pixels.
 *   points [N,2] float32 (x, y); values [N,C] float32
 *   pix    [n_pix] row-major pixel indices, or NULL for all H*W pixels
 * Outputs (each may be NULL), indexed by position in the pixel list:
 *   out     [n_pix, C]  c(q)
 *   den     [n_pix]     exact: Z' = sum_i exp(-(d_i^2 - m)/(2 sigma^2)) (>= 1)
 *                       truncated: Z = sum_{d_i <= k sigma} exp(-d_i^2/(2 sigma^2))
 *   shift   [n_pix]     exact: m = min_i d_i^2 ; truncated: 0
 *   skipped [n_pix]     exact: share of Z' carried by points with
 *                       d_i^2 > m + k^2 sigma^2 (what a radius rule drops);
 *                       truncated: share of the in-disc weight carried by
 *                       points whose inclusion is decided within rounding
 *                       (|d^2 - k^2 sigma^2| <= 1e-5 k^2 sigma^2)
 *   pairs   [n_pix]     exact: #{i : d_i^2 <= m + k^2 sigma^2};
 *                       truncated: #{i : d_i^2 <= k^2 sigma^2}
 * Returns 0, or -1 on invalid arguments.
 */
int oracle_forward(const float* points, const float* values, int64_t N, int C,
                   int64_t H, int64_t W, double sigma, int mode, double k,
                   const int64_t* pix, int64_t n_pix,
                   double* out, double* den, double* shift, double* skipped,
                   int64_t* pairs) {
    if (N < 0 || C < 1 || H < 1 || W < 1 || !(sigma > 0) || !(k > 0)) return -1;
    if (mode != ORACLE_EXACT && mode != ORACLE_TRUNCATED) return -1;
    if (pix == NULL) n_pix = H * W;
    const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
    const double r2 = k * k * sigma * sigma;

#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < n_pix; ++t) {
        int64_t p = pix ? pix[t] : t;
        double qx, qy;
        pixel_centre(p, W, &qx, &qy);
        double num[8];
        double* acc = C <= 8 ? num : (double*)calloc((size_t)C, sizeof(double));
        for (int c = 0; c < C; ++c) acc[c] = 0.0;
        double z = 0.0, m = 0.0, skip = 0.0;
        int64_t cnt = 0;
        if (N > 0 && mode == ORACLE_EXACT) {
            m = INFINITY;
            for (int64_t i = 0; i < N; ++i) {
                double d2 = sqdist(points, i, qx, qy);
                if (d2 < m) m = d2;
            }
            for (int64_t i = 0; i < N; ++i) {
                double d2 = sqdist(points, i, qx, qy);
                double w = exp(-(d2 - m) * inv2s2);
                z += w;
                for (int c = 0; c < C; ++c) acc[c] += w * (double)values[i * C + c];
                if (d2 <= m + r2) ++cnt; else skip += w;
            }
            for (int c = 0; c < C; ++c) acc[c] /= z;
            skip /= z;
        } else if (N > 0) {
            double amb = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                double d2 = sqdist(points, i, qx, qy);
                if (fabs(d2 - r2) <= 1e-5 * r2) amb += exp(-d2 * inv2s2);
                if (d2 > r2) continue;
                double w = exp(-d2 * inv2s2);
                z += w;
                ++cnt;
                for (int c = 0; c < C; ++c) acc[c] += w * (double)values[i * C + c];
            }
            if (z > 0) {
                for (int c = 0; c < C; ++c) acc[c] /= z;
                skip = amb / z;
            } else {
                for (int c = 0; c < C; ++c) acc[c] = 0.0;
                skip = amb > 0 ? 1.0 : 0.0;
            }
        }
        if (out)
            for (int c = 0; c < C; ++c) out[t * C + c] = acc[c];
        if (den) den[t] = z;
        if (shift) shift[t] = m;
        if (skipped) skipped[t] = skip;
        if (pairs) pairs[t] = cnt;
        if (acc != num) free(acc);
    }
    return 0;
}

/*
 * Backward pass: gradients of L = sum_q sum_c g_c(q) c_c(q) with respect to
 * the point positions, the point values and sigma (chain rule on Eq. 1; see
 * the header).  grad [H,W,C] float32 is the upstream gradient dL/dc.
 * Outputs (each may be NULL): gpoints [N,2], gvalues [N,C], gsigma [1].
 * O(N*H*W); meant for small cases.
 */
int oracle_backward(const float* points, const float* values, int64_t N, int C,
                    int64_t H, int64_t W, double sigma, int mode, double k,
                    const float* grad, double* gpoints, double* gvalues,
                    double* gsigma) {
    if (N < 0 || C < 1 || C > 8 || H < 1 || W < 1 || !(sigma > 0) || !(k > 0)) return -1;
    if (mode != ORACLE_EXACT && mode != ORACLE_TRUNCATED) return -1;
    const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
    const double s2 = sigma * sigma, s3 = s2 * sigma;
    const double r2 = k * k * sigma * sigma;
    const int64_t P = H * W;
    int nt = oracle_num_threads();
    size_t per = (size_t)N * (size_t)(2 + C) + 1;
    double* part = (double*)calloc(per * (size_t)nt, sizeof(double));
    double* wbuf_all = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1) * (size_t)nt);
    if (!part || !wbuf_all) { free(part); free(wbuf_all); return -2; }

#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* acc = part + per * (size_t)tid;   /* [N*2 | N*C | 1] */
        double* w = wbuf_all + (size_t)(N > 0 ? N : 1) * (size_t)tid;
        double chat[8], G[8];
#pragma omp for schedule(dynamic, 16)
        for (int64_t p = 0; p < P; ++p) {
            if (N == 0) continue;
            int any = 0;   /* pixels with a zero upstream gradient contribute nothing */
            for (int c = 0; c < C; ++c) any |= grad[p * C + c] != 0.0f;
            if (!any) continue;
            double qx, qy;
            pixel_centre(p, W, &qx, &qy);
            double m = 0.0;
            if (mode == ORACLE_EXACT) {
                m = INFINITY;
                for (int64_t i = 0; i < N; ++i) {
                    double d2 = sqdist(points, i, qx, qy);
                    if (d2 < m) m = d2;
                }
            }
            double z = 0.0;
            for (int c = 0; c < C; ++c) chat[c] = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                double d2 = sqdist(points, i, qx, qy);
                double wi = (mode == ORACLE_TRUNCATED && d2 > r2) ? 0.0 : exp(-(d2 - m) * inv2s2);
                w[i] = wi;
                z += wi;
                for (int c = 0; c < C; ++c) chat[c] += wi * (double)values[i * C + c];
            }
            if (!(z > 0)) continue;  /* truncated pixel with no point: constant 0 */
            for (int c = 0; c < C; ++c) {
                chat[c] /= z;
                G[c] = (double)grad[p * C + c] / z;
            }
            for (int64_t i = 0; i < N; ++i) {
                if (w[i] == 0.0) continue;
                double t = 0.0;
                for (int c = 0; c < C; ++c) {
                    acc[2 * N + i * C + c] += w[i] * G[c];
                    t += G[c] * ((double)values[i * C + c] - chat[c]);
                }
                double dx = qx - (double)points[2 * i];
                double dy = qy - (double)points[2 * i + 1];
                double wt = w[i] * t;
                acc[2 * i] += wt * dx / s2;
                acc[2 * i + 1] += wt * dy / s2;
                acc[(size_t)N * (2 + C)] += wt * (dx * dx + dy * dy) / s3;
            }
        }
    }
    for (size_t e = 0; e < per; ++e) {
        double s = 0.0;
        for (int t = 0; t < nt; ++t) s += part[per * (size_t)t + e];
        part[e] = s;
    }
    if (gpoints) memcpy(gpoints, part, sizeof(double) * (size_t)N * 2);
    if (gvalues) memcpy(gvalues, part + 2 * N, sizeof(double) * (size_t)N * (size_t)C);
    if (gsigma) *gsigma = part[(size_t)N * (2 + C)];
    free(part);
    free(wbuf_all);
    return 0;
}

/*
 * Per-point sigma: an extension the paper does not make (its section 2
 * fixes one sigma for all points).  Point i is the normal N(mu_i,
 * sigma_i^2 I), and its normaliser 1/(2 pi sigma_i^2) no longer cancels in
 * Eq. 1; with the common 1/(2 pi) cancelled,
 *     w_i(q) = exp(-d_i^2 / (2 sigma_i^2)) / sigma_i^2,
 *     c(q)   = sum_i w_i c_i / sum_i w_i .
 * EXACT: all points, evaluated relative to the largest weight at q:
 *   w_i / w_max = exp(ln w_i - L), L = max_i ln w_i (no underflow);
 *   den = sum_i w_i / w_max (>= 1), shift = L.
 * TRUNCATED: only points with d_i <= k sigma_i, weights unshifted;
 *   den = sum of those w_i, shift 0; skipped = share of the in-disc weight
 *   carried by points within rounding of their radius
 *   (|d_i^2 - k^2 sigma_i^2| <= 1e-5 k^2 sigma_i^2); pairs counts the points
 *   inside their radius.
 * sigmas [N] float32, each > 0.  Returns 0, or -1 on invalid arguments.
 */
static double log_weight_pp(double d2, double s) { return -d2 / (2.0 * s * s) - 2.0 * log(s); }

int oracle_forward_pp(const float* points, const float* values, const float* sigmas, int64_t N, int C,
                      int64_t H, int64_t W, int mode, double k, const int64_t* pix, int64_t n_pix,
                      double* out, double* den, double* shift, double* skipped, int64_t* pairs) {
    if (N < 0 || C < 1 || H < 1 || W < 1 || !(k > 0) || (N > 0 && !sigmas)) return -1;
    if (mode != ORACLE_EXACT && mode != ORACLE_TRUNCATED) return -1;
    for (int64_t i = 0; i < N; ++i)
        if (!((double)sigmas[i] > 0)) return -1;
    if (pix == NULL) n_pix = H * W;

#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < n_pix; ++t) {
        int64_t p = pix ? pix[t] : t;
        double qx, qy;
        pixel_centre(p, W, &qx, &qy);
        double num[8];
        double* acc = C <= 8 ? num : (double*)calloc((size_t)C, sizeof(double));
        for (int c = 0; c < C; ++c) acc[c] = 0.0;
        double z = 0.0, L = 0.0, skip = 0.0;
        int64_t cnt = 0;
        if (N > 0 && mode == ORACLE_EXACT) {
            L = -INFINITY;
            for (int64_t i = 0; i < N; ++i) {
                double lw = log_weight_pp(sqdist(points, i, qx, qy), (double)sigmas[i]);
                if (lw > L) L = lw;
            }
            for (int64_t i = 0; i < N; ++i) {
                double w = exp(log_weight_pp(sqdist(points, i, qx, qy), (double)sigmas[i]) - L);
                z += w;
                ++cnt;
                for (int c = 0; c < C; ++c) acc[c] += w * (double)values[i * C + c];
            }
            for (int c = 0; c < C; ++c) acc[c] /= z;
        } else if (N > 0) {
            double amb = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                double s = (double)sigmas[i];
                double d2 = sqdist(points, i, qx, qy);
                double r2 = k * k * s * s;
                if (fabs(d2 - r2) <= 1e-5 * r2) amb += exp(log_weight_pp(d2, s));
                if (d2 > r2) continue;
                double w = exp(log_weight_pp(d2, s));
                z += w;
                ++cnt;
                for (int c = 0; c < C; ++c) acc[c] += w * (double)values[i * C + c];
            }
            if (z > 0) {
                for (int c = 0; c < C; ++c) acc[c] /= z;
                skip = amb / z;
            } else {
                for (int c = 0; c < C; ++c) acc[c] = 0.0;
                skip = amb > 0 ? 1.0 : 0.0;
            }
        }
        if (out)
            for (int c = 0; c < C; ++c) out[t * C + c] = acc[c];
        if (den) den[t] = z;
        if (shift) shift[t] = L;
        if (skipped) skipped[t] = skip;
        if (pairs) pairs[t] = cnt;
        if (acc != num) free(acc);
    }
    return 0;
}

/*
 * Backward pass with per-point sigma: gradients of L = sum_q sum_c g_c(q)
 * c_c(q) with respect to the positions, values and per-point sigmas.  With
 * t_i(q) = sum_c (g_c(q) / Z_q) (c_{i,c} - c_c(q)) and the chain rule on
 * the per-point Eq. 1 (d ln w_i / d mu_i = (q - mu_i) / sigma_i^2,
 * d ln w_i / d sigma_i = d_i^2 / sigma_i^3 - 2 / sigma_i):
 *     dL/dc_{i,c}   = sum_q (w_i / Z_q) g_c(q)
 *     dL/dmu_i      = sum_q (w_i / Z_q) t_i(q) (q - mu_i) / sigma_i^2
 *     dL/dsigma_i   = sum_q (w_i / Z_q) t_i(q) (d_i^2 / sigma_i^3 - 2 / sigma_i)
 * Outputs (each may be NULL): gpoints [N,2], gvalues [N,C], gsigmas [N].
 */
int oracle_backward_pp(const float* points, const float* values, const float* sigmas, int64_t N, int C,
                       int64_t H, int64_t W, int mode, double k, const float* grad, double* gpoints,
                       double* gvalues, double* gsigmas) {
    if (N < 0 || C < 1 || C > 8 || H < 1 || W < 1 || !(k > 0) || (N > 0 && !sigmas)) return -1;
    if (mode != ORACLE_EXACT && mode != ORACLE_TRUNCATED) return -1;
    for (int64_t i = 0; i < N; ++i)
        if (!((double)sigmas[i] > 0)) return -1;
    const int64_t P = H * W;
    int nt = oracle_num_threads();
    size_t per = (size_t)N * (size_t)(3 + C) + 1;
    double* part = (double*)calloc(per * (size_t)nt, sizeof(double));
    double* wbuf_all = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1) * (size_t)nt);
    if (!part || !wbuf_all) { free(part); free(wbuf_all); return -2; }

#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* acc = part + per * (size_t)tid;   /* [N*2 | N*C | N] */
        double* w = wbuf_all + (size_t)(N > 0 ? N : 1) * (size_t)tid;
        double chat[8], G[8];
#pragma omp for schedule(dynamic, 16)
        for (int64_t p = 0; p < P; ++p) {
            if (N == 0) continue;
            int any = 0;
            for (int c = 0; c < C; ++c) any |= grad[p * C + c] != 0.0f;
            if (!any) continue;
            double qx, qy;
            pixel_centre(p, W, &qx, &qy);
            double L = 0.0;
            if (mode == ORACLE_EXACT) {
                L = -INFINITY;
                for (int64_t i = 0; i < N; ++i) {
                    double lw = log_weight_pp(sqdist(points, i, qx, qy), (double)sigmas[i]);
                    if (lw > L) L = lw;
                }
            }
            double z = 0.0;
            for (int c = 0; c < C; ++c) chat[c] = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                double s = (double)sigmas[i];
                double d2 = sqdist(points, i, qx, qy);
                double wi = (mode == ORACLE_TRUNCATED && d2 > k * k * s * s) ? 0.0 : exp(log_weight_pp(d2, s) - L);
                w[i] = wi;
                z += wi;
                for (int c = 0; c < C; ++c) chat[c] += wi * (double)values[i * C + c];
            }
            if (!(z > 0)) continue;
            for (int c = 0; c < C; ++c) {
                chat[c] /= z;
                G[c] = (double)grad[p * C + c] / z;
            }
            for (int64_t i = 0; i < N; ++i) {
                if (w[i] == 0.0) continue;
                double s = (double)sigmas[i];
                double t = 0.0;
                for (int c = 0; c < C; ++c) {
                    acc[2 * N + i * C + c] += w[i] * G[c];
                    t += G[c] * ((double)values[i * C + c] - chat[c]);
                }
                double dx = qx - (double)points[2 * i];
                double dy = qy - (double)points[2 * i + 1];
                double wt = w[i] * t;
                acc[2 * i] += wt * dx / (s * s);
                acc[2 * i + 1] += wt * dy / (s * s);
                acc[(size_t)N * (2 + C) + i] += wt * ((dx * dx + dy * dy) / (s * s * s) - 2.0 / s);
            }
        }
    }
    for (size_t e = 0; e < per; ++e) {
        double s = 0.0;
        for (int t = 0; t < nt; ++t) s += part[per * (size_t)t + e];
        part[e] = s;
    }
    if (gpoints) memcpy(gpoints, part, sizeof(double) * (size_t)N * 2);
    if (gvalues) memcpy(gvalues, part + 2 * N, sizeof(double) * (size_t)N * (size_t)C);
    if (gsigmas) memcpy(gsigmas, part + (size_t)N * (2 + C), sizeof(double) * (size_t)N);
    free(part);
    free(wbuf_all);
    return 0;
}

/*
 * Anisotropic (axis-aligned) extension: point i is N(mu_i, diag(sx_i^2,
 * sy_i^2)).  Its normaliser 1/(2 pi sx_i sy_i) is kept; with the common
 * 1/(2 pi) cancelled,
 *     ln w_i(q) = -dx^2 / (2 sx_i^2) - dy^2 / (2 sy_i^2) - ln sx_i - ln sy_i,
 *     c(q) = sum_i w_i c_i / sum_i w_i                          (Eq. 1)
 * dx = qx - x_i, dy = qy - y_i.  EXACT: all points, relative to the largest
 * weight at q (den >= 1, shift = L = max ln w_i).  TRUNCATED: only points
 * inside their ellipse, dx^2/sx^2 + dy^2/sy^2 <= k^2, unshifted; skipped and
 * pairs as for oracle_forward_pp (the ellipse's Mahalanobis radius in place
 * of d^2 <= k^2 sigma^2).  sigmas_xy [N,2] = (sx, sy), each > 0.
 */
static double maha2(double dx, double dy, double sx, double sy) { return dx * dx / (sx * sx) + dy * dy / (sy * sy); }
static double log_weight_an(double dx, double dy, double sx, double sy) {
    return -0.5 * maha2(dx, dy, sx, sy) - log(sx) - log(sy);
}

int oracle_forward_aniso(const float* points, const float* values, const float* sigmas_xy, int64_t N, int C,
                         int64_t H, int64_t W, int mode, double k, const int64_t* pix, int64_t n_pix,
                         double* out, double* den, double* shift, double* skipped, int64_t* pairs) {
    if (N < 0 || C < 1 || H < 1 || W < 1 || !(k > 0) || (N > 0 && !sigmas_xy)) return -1;
    if (mode != ORACLE_EXACT && mode != ORACLE_TRUNCATED) return -1;
    for (int64_t i = 0; i < 2 * N; ++i)
        if (!((double)sigmas_xy[i] > 0)) return -1;
    if (pix == NULL) n_pix = H * W;

#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < n_pix; ++t) {
        int64_t p = pix ? pix[t] : t;
        double qx, qy;
        pixel_centre(p, W, &qx, &qy);
        double num[8];
        double* acc = C <= 8 ? num : (double*)calloc((size_t)C, sizeof(double));
        for (int c = 0; c < C; ++c) acc[c] = 0.0;
        double z = 0.0, L = 0.0, skip = 0.0;
        int64_t cnt = 0;
        if (N > 0 && mode == ORACLE_EXACT) {
            L = -INFINITY;
            for (int64_t i = 0; i < N; ++i) {
                double lw = log_weight_an(qx - (double)points[2 * i], qy - (double)points[2 * i + 1],
                                          (double)sigmas_xy[2 * i], (double)sigmas_xy[2 * i + 1]);
                if (lw > L) L = lw;
            }
            for (int64_t i = 0; i < N; ++i) {
                double w = exp(log_weight_an(qx - (double)points[2 * i], qy - (double)points[2 * i + 1],
                                             (double)sigmas_xy[2 * i], (double)sigmas_xy[2 * i + 1]) - L);
                z += w;
                ++cnt;
                for (int c = 0; c < C; ++c) acc[c] += w * (double)values[i * C + c];
            }
            for (int c = 0; c < C; ++c) acc[c] /= z;
        } else if (N > 0) {
            double amb = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                double sx = (double)sigmas_xy[2 * i], sy = (double)sigmas_xy[2 * i + 1];
                double dx = qx - (double)points[2 * i], dy = qy - (double)points[2 * i + 1];
                double m2 = maha2(dx, dy, sx, sy);
                double r2 = k * k;
                if (fabs(m2 - r2) <= 1e-5 * r2) amb += exp(log_weight_an(dx, dy, sx, sy));
                if (m2 > r2) continue;
                double w = exp(log_weight_an(dx, dy, sx, sy));
                z += w;
                ++cnt;
                for (int c = 0; c < C; ++c) acc[c] += w * (double)values[i * C + c];
            }
            if (z > 0) {
                for (int c = 0; c < C; ++c) acc[c] /= z;
                skip = amb / z;
            } else {
                for (int c = 0; c < C; ++c) acc[c] = 0.0;
                skip = amb > 0 ? 1.0 : 0.0;
            }
        }
        if (out)
            for (int c = 0; c < C; ++c) out[t * C + c] = acc[c];
        if (den) den[t] = z;
        if (shift) shift[t] = L;
        if (skipped) skipped[t] = skip;
        if (pairs) pairs[t] = cnt;
        if (acc != num) free(acc);
    }
    return 0;
}

/*
 * Backward pass of the anisotropic extension, by the chain rule on Eq. 1:
 * with t_i(q) = sum_c (g_c(q) / Z_q) (c_{i,c} - c_c(q)),
 *   d ln w_i / d x_i  = dx / sx_i^2,      d ln w_i / d y_i  = dy / sy_i^2,
 *   d ln w_i / d sx_i = dx^2 / sx_i^3 - 1 / sx_i,
 *   d ln w_i / d sy_i = dy^2 / sy_i^3 - 1 / sy_i,
 * and every gradient is sum_q (w_i / Z_q) t_i(q) times that factor
 * (dL/dc_{i,c} = sum_q (w_i / Z_q) g_c(q)).
 * Outputs (each may be NULL): gpoints [N,2], gvalues [N,C], gsigmas_xy [N,2].
 */
int oracle_backward_aniso(const float* points, const float* values, const float* sigmas_xy, int64_t N, int C,
                          int64_t H, int64_t W, int mode, double k, const float* grad, double* gpoints,
                          double* gvalues, double* gsigmas_xy) {
    if (N < 0 || C < 1 || C > 8 || H < 1 || W < 1 || !(k > 0) || (N > 0 && !sigmas_xy)) return -1;
    if (mode != ORACLE_EXACT && mode != ORACLE_TRUNCATED) return -1;
    for (int64_t i = 0; i < 2 * N; ++i)
        if (!((double)sigmas_xy[i] > 0)) return -1;
    const int64_t P = H * W;
    int nt = oracle_num_threads();
    size_t per = (size_t)N * (size_t)(4 + C) + 1;
    double* part = (double*)calloc(per * (size_t)nt, sizeof(double));
    double* wbuf_all = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1) * (size_t)nt);
    if (!part || !wbuf_all) { free(part); free(wbuf_all); return -2; }

#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* acc = part + per * (size_t)tid;   /* [N*2 | N*C | N*2] */
        double* w = wbuf_all + (size_t)(N > 0 ? N : 1) * (size_t)tid;
        double chat[8], G[8];
#pragma omp for schedule(dynamic, 16)
        for (int64_t p = 0; p < P; ++p) {
            if (N == 0) continue;
            int any = 0;
            for (int c = 0; c < C; ++c) any |= grad[p * C + c] != 0.0f;
            if (!any) continue;
            double qx, qy;
            pixel_centre(p, W, &qx, &qy);
            double L = 0.0;
            if (mode == ORACLE_EXACT) {
                L = -INFINITY;
                for (int64_t i = 0; i < N; ++i) {
                    double lw = log_weight_an(qx - (double)points[2 * i], qy - (double)points[2 * i + 1],
                                              (double)sigmas_xy[2 * i], (double)sigmas_xy[2 * i + 1]);
                    if (lw > L) L = lw;
                }
            }
            double z = 0.0;
            for (int c = 0; c < C; ++c) chat[c] = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                double sx = (double)sigmas_xy[2 * i], sy = (double)sigmas_xy[2 * i + 1];
                double dx = qx - (double)points[2 * i], dy = qy - (double)points[2 * i + 1];
                double wi = (mode == ORACLE_TRUNCATED && maha2(dx, dy, sx, sy) > k * k)
                                ? 0.0 : exp(log_weight_an(dx, dy, sx, sy) - L);
                w[i] = wi;
                z += wi;
                for (int c = 0; c < C; ++c) chat[c] += wi * (double)values[i * C + c];
            }
            if (!(z > 0)) continue;
            for (int c = 0; c < C; ++c) {
                chat[c] /= z;
                G[c] = (double)grad[p * C + c] / z;
            }
            for (int64_t i = 0; i < N; ++i) {
                if (w[i] == 0.0) continue;
                double sx = (double)sigmas_xy[2 * i], sy = (double)sigmas_xy[2 * i + 1];
                double t = 0.0;
                for (int c = 0; c < C; ++c) {
                    acc[2 * N + i * C + c] += w[i] * G[c];
                    t += G[c] * ((double)values[i * C + c] - chat[c]);
                }
                double dx = qx - (double)points[2 * i];
                double dy = qy - (double)points[2 * i + 1];
                double wt = w[i] * t;
                double* gs = acc + (size_t)N * (2 + C);
                acc[2 * i] += wt * dx / (sx * sx);
                acc[2 * i + 1] += wt * dy / (sy * sy);
                gs[2 * i] += wt * (dx * dx / (sx * sx * sx) - 1.0 / sx);
                gs[2 * i + 1] += wt * (dy * dy / (sy * sy * sy) - 1.0 / sy);
            }
        }
    }
    for (size_t e = 0; e < per; ++e) {
        double s = 0.0;
        for (int t = 0; t < nt; ++t) s += part[per * (size_t)t + e];
        part[e] = s;
    }
    if (gpoints) memcpy(gpoints, part, sizeof(double) * (size_t)N * 2);
    if (gvalues) memcpy(gvalues, part + 2 * N, sizeof(double) * (size_t)N * (size_t)C);
    if (gsigmas_xy) memcpy(gsigmas_xy, part + (size_t)N * (2 + C), sizeof(double) * (size_t)N * 2);
    free(part);
    free(wbuf_all);
    return 0;
}

/*
 * Full-covariance extension: point i is N(mu_i, S_i) with
 *     S_i = [[sx^2, rho sx sy], [rho sx sy, sy^2]],  |rho| < 1,
 * and its normaliser 1/(2 pi sqrt(det S_i)) = 1/(2 pi sx sy sqrt(1 - rho^2))
 * kept.  With d = q - mu_i and the quadratic form
 *     Q = d^T S_i^-1 d = (dx^2/sx^2 - 2 rho dx dy/(sx sy) + dy^2/sy^2) / (1 - rho^2),
 *     ln w_i(q) = -Q/2 - ln sx - ln sy - ln(1 - rho^2)/2,
 *     c(q) = sum_i w_i c_i / sum_i w_i                          (Eq. 1)
 * EXACT / TRUNCATED (Q <= k^2) and the outputs as for oracle_forward_aniso.
 * cov [N,3] = (sx, sy, rho) per point, sx, sy > 0, |rho| < 1.
 */
static double quad_cov(double dx, double dy, const float* cv) {
    double sx = (double)cv[0], sy = (double)cv[1], r = (double)cv[2];
    return (dx * dx / (sx * sx) - 2.0 * r * dx * dy / (sx * sy) + dy * dy / (sy * sy)) / (1.0 - r * r);
}
static double log_norm_cov(const float* cv) {
    double sx = (double)cv[0], sy = (double)cv[1], r = (double)cv[2];
    return -log(sx) - log(sy) - 0.5 * log(1.0 - r * r);
}
static int cov_valid(const float* cov, int64_t N) {
    for (int64_t i = 0; i < N; ++i) {
        double sx = (double)cov[3 * i], sy = (double)cov[3 * i + 1], r = (double)cov[3 * i + 2];
        if (!(sx > 0) || !(sy > 0) || !(fabs(r) < 1.0)) return 0;
    }
    return 1;
}

int oracle_forward_cov(const float* points, const float* values, const float* cov, int64_t N, int C,
                       int64_t H, int64_t W, int mode, double k, const int64_t* pix, int64_t n_pix,
                       double* out, double* den, double* shift, double* skipped, int64_t* pairs) {
    if (N < 0 || C < 1 || H < 1 || W < 1 || !(k > 0) || (N > 0 && !cov)) return -1;
    if (mode != ORACLE_EXACT && mode != ORACLE_TRUNCATED) return -1;
    if (!cov_valid(cov, N)) return -1;
    if (pix == NULL) n_pix = H * W;

#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < n_pix; ++t) {
        int64_t p = pix ? pix[t] : t;
        double qx, qy;
        pixel_centre(p, W, &qx, &qy);
        double num[8];
        double* acc = C <= 8 ? num : (double*)calloc((size_t)C, sizeof(double));
        for (int c = 0; c < C; ++c) acc[c] = 0.0;
        double z = 0.0, L = 0.0, skip = 0.0;
        int64_t cnt = 0;
        if (N > 0 && mode == ORACLE_EXACT) {
            L = -INFINITY;
            for (int64_t i = 0; i < N; ++i) {
                double lw = -0.5 * quad_cov(qx - (double)points[2 * i], qy - (double)points[2 * i + 1], cov + 3 * i)
                            + log_norm_cov(cov + 3 * i);
                if (lw > L) L = lw;
            }
            for (int64_t i = 0; i < N; ++i) {
                double lw = -0.5 * quad_cov(qx - (double)points[2 * i], qy - (double)points[2 * i + 1], cov + 3 * i)
                            + log_norm_cov(cov + 3 * i);
                double w = exp(lw - L);
                z += w;
                ++cnt;
                for (int c = 0; c < C; ++c) acc[c] += w * (double)values[i * C + c];
            }
            for (int c = 0; c < C; ++c) acc[c] /= z;
        } else if (N > 0) {
            double amb = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                double Q = quad_cov(qx - (double)points[2 * i], qy - (double)points[2 * i + 1], cov + 3 * i);
                double r2 = k * k;
                double lw = -0.5 * Q + log_norm_cov(cov + 3 * i);
                if (fabs(Q - r2) <= 1e-5 * r2) amb += exp(lw);
                if (Q > r2) continue;
                double w = exp(lw);
                z += w;
                ++cnt;
                for (int c = 0; c < C; ++c) acc[c] += w * (double)values[i * C + c];
            }
            if (z > 0) {
                for (int c = 0; c < C; ++c) acc[c] /= z;
                skip = amb / z;
            } else {
                for (int c = 0; c < C; ++c) acc[c] = 0.0;
                skip = amb > 0 ? 1.0 : 0.0;
            }
        }
        if (out)
            for (int c = 0; c < C; ++c) out[t * C + c] = acc[c];
        if (den) den[t] = z;
        if (shift) shift[t] = L;
        if (skipped) skipped[t] = skip;
        if (pairs) pairs[t] = cnt;
        if (acc != num) free(acc);
    }
    return 0;
}

/*
 * Backward pass of the full-covariance extension, by the chain rule on
 * Eq. 1.  With m = dx dy / (sx sy) and e = 1 - rho^2:
 *   d ln w / d mu   = S^-1 d
 *   d ln w / d sx   = (dx^2/sx^3 - rho dx dy/(sx^2 sy)) / e - 1/sx
 *   d ln w / d sy   = (dy^2/sy^3 - rho dx dy/(sx sy^2)) / e - 1/sy
 *   d ln w / d rho  = (m - rho Q) / e + rho / e
 * each gradient being sum_q (w_i / Z_q) t_i(q) times that factor, t_i as for
 * oracle_backward_pp.  Outputs (each may be NULL): gpoints [N,2], gvalues
 * [N,C], gcov [N,3] = d/d(sx, sy, rho).
 */
int oracle_backward_cov(const float* points, const float* values, const float* cov, int64_t N, int C,
                        int64_t H, int64_t W, int mode, double k, const float* grad, double* gpoints,
                        double* gvalues, double* gcov) {
    if (N < 0 || C < 1 || C > 8 || H < 1 || W < 1 || !(k > 0) || (N > 0 && !cov)) return -1;
    if (mode != ORACLE_EXACT && mode != ORACLE_TRUNCATED) return -1;
    if (!cov_valid(cov, N)) return -1;
    const int64_t P = H * W;
    int nt = oracle_num_threads();
    size_t per = (size_t)N * (size_t)(5 + C) + 1;
    double* part = (double*)calloc(per * (size_t)nt, sizeof(double));
    double* wbuf_all = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1) * (size_t)nt);
    if (!part || !wbuf_all) { free(part); free(wbuf_all); return -2; }

#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* acc = part + per * (size_t)tid;   /* [N*2 | N*C | N*3] */
        double* w = wbuf_all + (size_t)(N > 0 ? N : 1) * (size_t)tid;
        double chat[8], G[8];
#pragma omp for schedule(dynamic, 16)
        for (int64_t p = 0; p < P; ++p) {
            if (N == 0) continue;
            int any = 0;
            for (int c = 0; c < C; ++c) any |= grad[p * C + c] != 0.0f;
            if (!any) continue;
            double qx, qy;
            pixel_centre(p, W, &qx, &qy);
            double L = 0.0;
            if (mode == ORACLE_EXACT) {
                L = -INFINITY;
                for (int64_t i = 0; i < N; ++i) {
                    double lw = -0.5 * quad_cov(qx - (double)points[2 * i], qy - (double)points[2 * i + 1],
                                                cov + 3 * i) + log_norm_cov(cov + 3 * i);
                    if (lw > L) L = lw;
                }
            }
            double z = 0.0;
            for (int c = 0; c < C; ++c) chat[c] = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                double Q = quad_cov(qx - (double)points[2 * i], qy - (double)points[2 * i + 1], cov + 3 * i);
                double wi = (mode == ORACLE_TRUNCATED && Q > k * k) ? 0.0
                                                                     : exp(-0.5 * Q + log_norm_cov(cov + 3 * i) - L);
                w[i] = wi;
                z += wi;
                for (int c = 0; c < C; ++c) chat[c] += wi * (double)values[i * C + c];
            }
            if (!(z > 0)) continue;
            for (int c = 0; c < C; ++c) {
                chat[c] /= z;
                G[c] = (double)grad[p * C + c] / z;
            }
            for (int64_t i = 0; i < N; ++i) {
                if (w[i] == 0.0) continue;
                double sx = (double)cov[3 * i], sy = (double)cov[3 * i + 1], r = (double)cov[3 * i + 2];
                double e = 1.0 - r * r;
                double t = 0.0;
                for (int c = 0; c < C; ++c) {
                    acc[2 * N + i * C + c] += w[i] * G[c];
                    t += G[c] * ((double)values[i * C + c] - chat[c]);
                }
                double dx = qx - (double)points[2 * i];
                double dy = qy - (double)points[2 * i + 1];
                double wt = w[i] * t;
                /* S^-1 = [[1/sx^2, -rho/(sx sy)], [-rho/(sx sy), 1/sy^2]] / e */
                double ix = (dx / (sx * sx) - r * dy / (sx * sy)) / e;
                double iy = (dy / (sy * sy) - r * dx / (sx * sy)) / e;
                double Q = quad_cov(dx, dy, cov + 3 * i);
                double m = dx * dy / (sx * sy);
                double* gc = acc + (size_t)N * (2 + C);
                acc[2 * i] += wt * ix;
                acc[2 * i + 1] += wt * iy;
                gc[3 * i] += wt * ((dx * dx / (sx * sx * sx) - r * dx * dy / (sx * sx * sy)) / e - 1.0 / sx);
                gc[3 * i + 1] += wt * ((dy * dy / (sy * sy * sy) - r * dx * dy / (sx * sy * sy)) / e - 1.0 / sy);
                gc[3 * i + 2] += wt * ((m - r * Q) / e + r / e);
            }
        }
    }
    for (size_t e = 0; e < per; ++e) {
        double s = 0.0;
        for (int t = 0; t < nt; ++t) s += part[per * (size_t)t + e];
        part[e] = s;
    }
    if (gpoints) memcpy(gpoints, part, sizeof(double) * (size_t)N * 2);
    if (gvalues) memcpy(gvalues, part + 2 * N, sizeof(double) * (size_t)N * (size_t)C);
    if (gcov) memcpy(gcov, part + (size_t)N * (2 + C), sizeof(double) * (size_t)N * 3);
    free(part);
    free(wbuf_all);
    return 0;
}
