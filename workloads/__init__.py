"""Seeded synthetic inputs for the Gaussian-mixture interpolation workloads.

This module only draws random numbers and lays them out; it contains none of
the interpolation arithmetic, so both the FP64 oracle and the CUDA path can be
fed from it without sharing any code with each other.

Conventions (the paper leaves them open, section 1): positions are in output
pixel units, ``points[:, 0]`` is x (column direction, along W) and
``points[:, 1]`` is y (row direction, along H); the output pixel (i, j) sits at
(j + 0.5, i + 0.5).  Everything is float32, row-major and contiguous.

Workloads (shapes follow the paper's upsampling use case, section 3.2, with
synthetic fields standing in for the ImageNet images, which are not used):

* ``small_uniform``      N=4096 uniform in [0,64)^2, 64x64x3, sigma=0.75
* ``upsample_1024``      512^2 jittered source grid -> 1024x1024x3, sigma=1.0,
                         values from a smooth random field
* ``batched_uneven``     64 images, sides log-uniform in [128,1024],
                         N = 0.25*H*W clustered points, sigma U[0.5,2]
* ``fwd_bwd_512``        16 images 512x512x3, 65536 clustered points each,
                         sigma=1.0, upstream gradient N(0,1)
* ``serving``            request stream: Poisson arrivals, sides log-uniform
                         in [64,2048], N = U[0.1,1]*H*W, uniform or clustered
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

__all__ = [
    "Image", "uniform_points", "clustered_points", "smooth_field",
    "small_uniform", "upsample_1024", "batched_uneven", "fwd_bwd_512",
    "fd_subcase", "serving_stream", "tiny_random", "field_params", "eval_field", "reconstruction_case",
]


@dataclasses.dataclass
class Image:
    """One interpolation problem: points[N,2], values[N,C], sigma, H, W."""
    points: np.ndarray
    values: np.ndarray
    sigma: float
    H: int
    W: int

    @property
    def N(self) -> int:
        return int(self.points.shape[0])

    @property
    def C(self) -> int:
        return int(self.values.shape[1])


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def uniform_points(rng: np.random.Generator, n: int, H: int, W: int) -> np.ndarray:
    """n positions uniform in [0,W) x [0,H)."""
    xy = np.empty((n, 2), dtype=np.float64)
    xy[:, 0] = rng.uniform(0.0, W, n)
    xy[:, 1] = rng.uniform(0.0, H, n)
    pts = _f32(xy)
    # float32 rounding can land exactly on the upper edge; keep [0, W) x [0, H)
    np.minimum(pts[:, 0], np.nextafter(np.float32(W), np.float32(0)), out=pts[:, 0])
    np.minimum(pts[:, 1], np.nextafter(np.float32(H), np.float32(0)), out=pts[:, 1])
    return pts


def clustered_points(rng: np.random.Generator, n: int, H: int, W: int,
                     n_clusters: int = 8) -> np.ndarray:
    """n positions from a mixture of isotropic 2D Gaussian clusters.

    Centres are uniform in the frame, each cluster's std is U[0.05, 0.2] of
    min(H, W), the mixture weights are Dirichlet(1); samples falling outside
    [0,W) x [0,H) are redrawn from the same cluster.
    """
    centres = np.stack([rng.uniform(0, W, n_clusters), rng.uniform(0, H, n_clusters)], 1)
    stds = rng.uniform(0.05, 0.2, n_clusters) * min(H, W)
    weights = rng.dirichlet(np.ones(n_clusters))
    labels = rng.choice(n_clusters, size=n, p=weights)
    out = np.empty((n, 2), dtype=np.float64)
    todo = np.arange(n)
    while todo.size:
        lab = labels[todo]
        cand = centres[lab] + rng.standard_normal((todo.size, 2)) * stds[lab, None]
        cand32 = cand.astype(np.float32)
        ok = (cand32[:, 0] >= 0) & (cand32[:, 0] < W) & (cand32[:, 1] >= 0) & (cand32[:, 1] < H)
        out[todo[ok]] = cand[ok]
        todo = todo[~ok]
    return _f32(out)


def field_params(rng: np.random.Generator, C: int, n_waves: int = 32, std: float = 0.25,
                 max_cycles: float = 8.0):
    """Random sinusoid parameters of a smooth field, per channel (u, v, phi, a):
    frequencies U[-max_cycles, max_cycles] cycles per period, phases U[0,2pi),
    amplitudes U[0,1] rescaled so the (unclipped) field has the given std."""
    params = []
    for _ in range(C):
        u = rng.uniform(-max_cycles, max_cycles, n_waves)
        v = rng.uniform(-max_cycles, max_cycles, n_waves)
        phi = rng.uniform(0, 2 * math.pi, n_waves)
        a = rng.uniform(0, 1, n_waves)
        a *= std / math.sqrt(0.5 * float(np.sum(a * a)))
        params.append((u, v, phi, a))
    return params


def eval_field(params, xy: np.ndarray, period: float) -> np.ndarray:
    """Per channel 0.5 + the sum of the sinusoids at positions xy[:, (x, y)],
    clipped to [0,1], float32 [n, C]."""
    x = xy[:, 0].astype(np.float64)
    y = xy[:, 1].astype(np.float64)
    out = np.empty((xy.shape[0], len(params)), dtype=np.float64)
    for c, (u, v, phi, a) in enumerate(params):
        f = np.full(x.shape, 0.5)
        for k in range(len(a)):
            f += a[k] * np.sin(2 * math.pi * (u[k] * x + v[k] * y) / period + phi[k])
        out[:, c] = f
    return _f32(np.clip(out, 0.0, 1.0))


def smooth_field(rng: np.random.Generator, xy: np.ndarray, C: int, period: float,
                 n_waves: int = 32, std: float = 0.25) -> np.ndarray:
    """Per channel: 0.5 + sum of n_waves random 2D sinusoids (frequencies
    U[-8,8] cycles per ``period`` pixels), clipped to [0,1]."""
    return eval_field(field_params(rng, C, n_waves, std), xy, period)


def small_uniform(seed: int = 1) -> Image:
    """N=4096 points uniform in [0,64)^2, RGB U[0,1], sigma=0.75, 64x64 output."""
    rng = np.random.default_rng(seed)
    pts = uniform_points(rng, 4096, 64, 64)
    vals = _f32(rng.uniform(0, 1, (4096, 3)))
    return Image(pts, vals, 0.75, 64, 64)


def upsample_1024(seed: int = 2, src: int = 512, factor: int = 2, C: int = 3,
                  sigma: float = 1.0) -> Image:
    """A src x src source grid upsampled by ``factor`` (default 512^2 -> 1024^2).

    Source sample (l, k) sits at the centre of its factor x factor block,
    (factor*l + factor/2, factor*k + factor/2), jittered by U[-0.5, 0.5] px on
    each axis; its colour is a smooth random field evaluated there.
    """
    rng = np.random.default_rng(seed)
    H = W = src * factor
    ly, lx = np.meshgrid(np.arange(src), np.arange(src), indexing="ij")
    base = np.stack([lx.ravel() * factor + factor / 2.0, ly.ravel() * factor + factor / 2.0], 1)
    jit = rng.uniform(-0.5, 0.5, base.shape)
    pts = _f32(base + jit)
    vals = smooth_field(rng, pts, C, period=float(W))
    return Image(pts, vals, sigma, H, W)


def reconstruction_case(factor: int, side: int = 768, C: int = 3, seed: int = 6, max_cycles: float = 24.0):
    """A smooth random field (up to ``max_cycles`` cycles across the image)
    seen at full resolution (side x side pixel centres: the truth) and point-
    sampled at the centres of the factor x factor blocks (the low-resolution
    image).  Returns (points [n,2] in full-resolution pixel units, values
    [n,C], low [side/f, side/f, C], truth [side, side, C]); the low-resolution
    pixel (l, k) sits at ((k + 0.5) f, (l + 0.5) f), which is where
    align_corners=False resampling places it too."""
    rng = np.random.default_rng(seed)
    params = field_params(rng, C, max_cycles=max_cycles)
    n = side // factor
    ly, lx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    pts = _f32(np.stack([(lx.ravel() + 0.5) * factor, (ly.ravel() + 0.5) * factor], 1))
    vals = eval_field(params, pts, float(side))
    yy, xx = np.meshgrid(np.arange(side) + 0.5, np.arange(side) + 0.5, indexing="ij")
    truth = eval_field(params, np.stack([xx.ravel(), yy.ravel()], 1), float(side)).reshape(side, side, C)
    return pts, vals, vals.reshape(n, n, C), truth


def _log_uniform_int(rng, lo, hi, size=None):
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size))).astype(np.int64)


def batched_uneven(seed: int = 3, B: int = 64, lo: int = 128, hi: int = 1024,
                   density: float = 0.25, C: int = 3) -> List[Image]:
    """B images with sides log-uniform in [lo, hi], N = density*H*W clustered
    points (8 clusters), RGB U[0,1], sigma U[0.5, 2.0] per image."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(B):
        H = int(_log_uniform_int(rng, lo, hi))
        W = int(_log_uniform_int(rng, lo, hi))
        n = int(round(density * H * W))
        pts = clustered_points(rng, n, H, W)
        vals = _f32(rng.uniform(0, 1, (n, C)))
        sigma = float(np.float32(rng.uniform(0.5, 2.0)))
        out.append(Image(pts, vals, sigma, H, W))
    return out


def fwd_bwd_512(seed: int = 4, B: int = 16, side: int = 512, n: int = 65536,
                C: int = 3, sigma: float = 1.0):
    """B images of side x side from n clustered points each, plus an upstream
    gradient g ~ N(0,1) of shape [B, side, side, C]."""
    rng = np.random.default_rng(seed)
    imgs = []
    for _ in range(B):
        pts = clustered_points(rng, n, side, side)
        vals = _f32(rng.uniform(0, 1, (n, C)))
        imgs.append(Image(pts, vals, sigma, side, side))
    grad = _f32(rng.standard_normal((B, side, side, C)))
    return imgs, grad


def fd_subcase(seed: int = 4, side: int = 32, n: int = 256, C: int = 3,
               sigma: float = 1.0):
    """Small clustered case for finite-difference gradient checks."""
    rng = np.random.default_rng(seed + 1000)
    pts = clustered_points(rng, n, side, side)
    vals = _f32(rng.uniform(0, 1, (n, C)))
    grad = _f32(rng.standard_normal((side, side, C)))
    return Image(pts, vals, sigma, side, side), grad


def point_sigmas(seed: int, n: int, lo: float, hi: float, axes: int = 1) -> np.ndarray:
    """Per-point sigmas, log-uniform in [lo, hi] (float32): shape [n], or
    [n, axes] with independent draws per axis."""
    rng = np.random.default_rng(seed)
    size = n if axes == 1 else (n, axes)
    return _f32(np.exp(rng.uniform(np.log(lo), np.log(hi), size)))

def point_cov(seed: int, n: int, lo: float, hi: float, rmax: float = 0.8) -> np.ndarray:
    """Per-point covariances (sx, sy, rho) [n, 3] (float32): sx, sy
    log-uniform in [lo, hi], rho uniform in [-rmax, rmax]."""
    rng = np.random.default_rng(seed)
    s = np.exp(rng.uniform(np.log(lo), np.log(hi), (n, 2)))
    return _f32(np.concatenate([s, rng.uniform(-rmax, rmax, (n, 1))], 1))


def cov_bound(cov) -> float:
    """The largest sqrt(lambda_max) over the covariances (sx, sy, rho) [n, 3]
    (float64, rounded up by a relative 1e-6): the search-radius bound a full
    covariance per point needs."""
    c = np.asarray(cov, np.float64).reshape(-1, 3)
    a, d, b = c[:, 0] ** 2, c[:, 1] ** 2, c[:, 2] * c[:, 0] * c[:, 1]
    lam = 0.5 * (a + d) + np.sqrt((0.5 * (a - d)) ** 2 + b * b)
    return float(np.sqrt(lam.max()) * (1 + 1e-6)) if c.shape[0] else 1.0

def tiny_random(seed: int, N: int, H: int, W: int, C: int = 3, sigma: float = 1.0,
                clustered: bool = False, margin: float = 0.0) -> Image:
    """Small random case; ``margin`` widens the position range beyond the frame
    so that some points fall outside it."""
    rng = np.random.default_rng(seed)
    if clustered:
        pts = clustered_points(rng, N, H, W)
    else:
        xy = np.stack([rng.uniform(-margin, W + margin, N), rng.uniform(-margin, H + margin, N)], 1)
        pts = _f32(xy)
    vals = _f32(rng.uniform(0, 1, (N, C)))
    return Image(pts, vals, float(np.float32(sigma)), H, W)


@dataclasses.dataclass
class Request:
    """One serving request: arrival time (s from stream start) and its image."""
    rid: int
    t_arrival: float
    H: int
    W: int
    N: int
    clustered: bool
    sigma: float
    seed: int

    def materialise(self, C: int = 3) -> Image:
        rng = np.random.default_rng(self.seed)
        if self.clustered:
            pts = clustered_points(rng, self.N, self.H, self.W)
        else:
            pts = uniform_points(rng, self.N, self.H, self.W)
        vals = _f32(rng.uniform(0, 1, (self.N, C)))
        return Image(pts, vals, self.sigma, self.H, self.W)


def serving_stream(seed: int = 5, n_requests: int = 10000, rate: float = 2000.0,
                   lo: int = 64, hi: int = 2048) -> List[Request]:
    """Request descriptors with Poisson arrivals at ``rate`` per second.

    Sides are log-uniform in [lo, hi] (independently for H and W), the point
    count is U[0.1, 1.0] * H * W, a fair coin picks uniform or clustered
    positions, sigma is U[0.5, 2.0].  Payloads are drawn lazily by
    ``Request.materialise`` from a per-request seed.
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, n_requests)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for r in range(n_requests):
        H = int(_log_uniform_int(rng, lo, hi))
        W = int(_log_uniform_int(rng, lo, hi))
        N = max(1, int(round(rng.uniform(0.1, 1.0) * H * W)))
        clustered = bool(rng.integers(0, 2))
        sigma = float(np.float32(rng.uniform(0.5, 2.0)))
        out.append(Request(r, float(t[r]), H, W, N, clustered, sigma,
                           int(rng.integers(0, 2**31 - 1))))
    return out
