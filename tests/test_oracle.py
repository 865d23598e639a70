"""Pins for the FP64 oracle (CPU only).

The oracle is checked against things other than itself:

* closed forms derived from Eq. 1 / Eq. 2: one point (the colour is that
  point's colour; Z is its Gaussian value), two points (a logistic sigmoid of
  the squared-distance difference, evaluated with ``scipy.special.expit``);
* invariants of Eq. 1: constant colours give a constant image, permutation
  invariance, linearity in the colours, convexity, translation covariance;
* limits that reduce to textbook or library routines: sigma -> 0 on the
  identity grid returns the input; sigma -> 0 on an odd-factor upsampling grid
  is nearest-neighbour upsampling (``np.repeat``); sigma -> 0 on random points
  is the k-d tree nearest neighbour (``scipy.spatial.cKDTree``); sigma -> inf
  gives the plain mean;
* the radius rule's pair count against a k-d tree ball count;
* the analytic gradient against FP64 central finite differences of the
  oracle's own forward, against torch autograd on an independent FP64 torch
  evaluation (the paper's own validation method, section 3.1, extended to the
  backward pass), and against the identity sum_i dL/dc_i = sum_q g(q).

Each pin is chosen so that a plausible mistake in the oracle (a dropped term,
a wrong sign, a swapped axis, a transposed operand) fails at least one test.
"""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree
from scipy.special import expit

import oracle
import workloads as wl


def _grid(H, W):
    yy, xx = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    return xx, yy


# ---------------------------------------------------------------- closed forms
def test_single_point_exact_closed_form():
    p = np.array([[3.25, 5.5]], np.float32)
    c = np.array([[0.2, 0.7, 0.9]], np.float32)
    H, W, s = 9, 7, 1.3
    r = oracle.forward(p, c, H, W, s)
    np.testing.assert_array_equal(r["image"], np.broadcast_to(c.astype(np.float64), (H, W, 3)))
    xx, yy = _grid(H, W)
    d2 = (xx - 3.25) ** 2 + (yy - 5.5) ** 2
    np.testing.assert_allclose(r["shift"], d2, rtol=0, atol=1e-12)
    # Z' is shifted by exp(m / 2 s^2): the unshifted Gaussian value is recovered
    np.testing.assert_allclose(r["den"] * np.exp(-r["shift"] / (2 * s * s)),
                               np.exp(-d2 / (2 * s * s)), rtol=1e-13)
    assert (r["pairs"] == 1).all()


def test_single_point_truncated_closed_form():
    p = np.array([[4.1, 2.9]], np.float32)
    c = np.array([[0.5, 0.25]], np.float32)
    H, W, s, k = 12, 10, 0.8, 3.0
    r = oracle.forward(p, c, H, W, s, mode=oracle.TRUNCATED, k=k)
    xx, yy = _grid(H, W)
    d2 = (xx - np.float64(np.float32(4.1))) ** 2 + (yy - np.float64(np.float32(2.9))) ** 2
    inside = d2 <= (k * s) ** 2
    assert inside.any() and (~inside).any()
    np.testing.assert_array_equal(r["image"][inside], np.broadcast_to(c.astype(np.float64), (inside.sum(), 2)))
    np.testing.assert_array_equal(r["image"][~inside], 0.0)
    np.testing.assert_allclose(r["den"][inside], np.exp(-d2[inside] / (2 * s * s)), rtol=1e-13)
    np.testing.assert_array_equal(r["den"][~inside], 0.0)


@pytest.mark.parametrize("s", [0.4, 1.0, 3.0])
def test_two_points_sigmoid(s):
    p = np.array([[2.3, 3.1], [6.7, 4.4]], np.float32)
    c = np.array([[0.1, 0.9], [0.8, 0.3]], np.float32)
    H, W = 8, 10
    r = oracle.forward(p, c, H, W, s)
    xx, yy = _grid(H, W)
    pf = p.astype(np.float64)
    d1 = (xx - pf[0, 0]) ** 2 + (yy - pf[0, 1]) ** 2
    d2 = (xx - pf[1, 0]) ** 2 + (yy - pf[1, 1]) ** 2
    lam = expit((d1 - d2) / (2 * s * s))       # weight share of point 2
    cf = c.astype(np.float64)
    ref = cf[0][None, None, :] + (cf[1] - cf[0])[None, None, :] * lam[..., None]
    np.testing.assert_allclose(r["image"], ref, rtol=0, atol=1e-14)


# ---------------------------------------------------------------- invariants
def test_constant_values_constant_image():
    im = wl.tiny_random(11, 50, 13, 17, C=3, sigma=0.9, margin=3.0)
    vals = np.full_like(im.values, 0.375)
    r = oracle.forward(im.points, vals, im.H, im.W, im.sigma)
    np.testing.assert_allclose(r["image"], 0.375, rtol=0, atol=1e-15)


def test_permutation_invariance():
    im = wl.tiny_random(12, 64, 16, 16, C=3, sigma=1.1)
    perm = np.random.default_rng(0).permutation(im.N)
    a = oracle.forward(im.points, im.values, im.H, im.W, im.sigma)
    b = oracle.forward(im.points[perm], im.values[perm], im.H, im.W, im.sigma)
    np.testing.assert_allclose(a["image"], b["image"], rtol=0, atol=1e-14)
    np.testing.assert_array_equal(a["shift"], b["shift"])


def test_linearity_in_values():
    im = wl.tiny_random(13, 40, 12, 14, C=2, sigma=0.7)
    rng = np.random.default_rng(1)
    # colours on a 2^-10 grid and power-of-two coefficients keep a*v1 + b*v2 exact
    v1 = (rng.integers(0, 1024, im.values.shape) / 1024.0).astype(np.float32)
    v2 = (rng.integers(0, 1024, im.values.shape) / 1024.0).astype(np.float32)
    a, b = 0.25, 0.5
    f1 = oracle.forward(im.points, v1, im.H, im.W, im.sigma)["image"]
    f2 = oracle.forward(im.points, v2, im.H, im.W, im.sigma)["image"]
    f12 = oracle.forward(im.points, (a * v1 + b * v2).astype(np.float32), im.H, im.W, im.sigma)["image"]
    np.testing.assert_allclose(f12, a * f1 + b * f2, rtol=0, atol=1e-14)


def test_convexity():
    im = wl.tiny_random(14, 30, 20, 20, C=3, sigma=2.0, margin=5.0)
    r = oracle.forward(im.points, im.values, im.H, im.W, im.sigma)
    lo = im.values.min(0).astype(np.float64)
    hi = im.values.max(0).astype(np.float64)
    assert (r["image"] >= lo - 1e-15).all() and (r["image"] <= hi + 1e-15).all()


def test_translation_covariance():
    im = wl.tiny_random(15, 60, 20, 24, C=3, sigma=1.2)
    dx, dy = 3, 2
    # positions on a 2^-12 grid so that the integer translation is exact in float32
    pts = (np.round(im.points * 4096) / 4096).astype(np.float32)
    sh = (pts + np.array([dx, dy], np.float32)).astype(np.float32)
    a = oracle.forward(pts, im.values, im.H, im.W, im.sigma)["image"]
    b = oracle.forward(sh, im.values, im.H, im.W, im.sigma)["image"]
    np.testing.assert_allclose(b[dy:, dx:], a[:-dy, :-dx], rtol=0, atol=1e-13)


def test_axis_convention():
    # one point far to the right (large x) must colour the right-hand columns
    p = np.array([[0.5, 0.5], [9.5, 0.5]], np.float32)
    c = np.array([[0.0], [1.0]], np.float32)
    r = oracle.forward(p, c, 2, 10, 0.5)["image"][..., 0]
    assert r[0, 9] > 0.99 and r[0, 0] < 0.01


# ---------------------------------------------------------------- limits
def test_identity_grid_small_sigma():
    H, W = 9, 11
    xx, yy = _grid(H, W)
    pts = np.stack([xx.ravel(), yy.ravel()], 1).astype(np.float32)
    vals = np.random.default_rng(2).uniform(0, 1, (H * W, 3)).astype(np.float32)
    r = oracle.forward(pts, vals, H, W, 1e-3)
    np.testing.assert_array_equal(r["image"].reshape(-1, 3), vals.astype(np.float64))


def test_odd_upsampling_is_nearest_neighbour():
    s, h, w = 3, 5, 6
    src = np.random.default_rng(3).uniform(0, 1, (h, w, 2)).astype(np.float32)
    ly, lx = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    pts = np.stack([s * (lx.ravel() + 0.5), s * (ly.ravel() + 0.5)], 1).astype(np.float32)
    r = oracle.forward(pts, src.reshape(-1, 2), h * s, w * s, 0.05)["image"]
    ref = np.repeat(np.repeat(src, s, axis=0), s, axis=1).astype(np.float64)
    np.testing.assert_allclose(r, ref, rtol=0, atol=1e-12)


def test_small_sigma_matches_kdtree_nearest_neighbour():
    im = wl.tiny_random(16, 80, 24, 24, C=3, sigma=0.02, margin=2.0)
    r = oracle.forward(im.points, im.values, im.H, im.W, im.sigma)
    xx, yy = _grid(im.H, im.W)
    q = np.stack([xx.ravel(), yy.ravel()], 1)
    d, idx = cKDTree(im.points.astype(np.float64)).query(q, k=2)
    gap = d[:, 1] ** 2 - d[:, 0] ** 2
    ok = gap > 0.05   # weight ratio exp(-gap / (2 s^2)) < 1e-27
    assert ok.mean() > 0.95
    np.testing.assert_allclose(r["image"].reshape(-1, 3)[ok], im.values[idx[ok, 0]].astype(np.float64),
                               rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["shift"].ravel(), d[:, 0] ** 2, rtol=1e-12, atol=1e-12)


def test_large_sigma_is_mean():
    im = wl.tiny_random(17, 40, 10, 10, C=3, sigma=1e4)
    r = oracle.forward(im.points, im.values, im.H, im.W, im.sigma)
    # every weight is within max d^2 / (2 s^2) of 1 relative
    err = (2 * 15.0 ** 2) / (2 * 1e8)
    np.testing.assert_allclose(r["image"], np.broadcast_to(im.values.mean(0, dtype=np.float64), r["image"].shape),
                               rtol=0, atol=err)


def test_truncated_equals_exact_when_all_points_inside():
    im = wl.tiny_random(18, 20, 6, 6, C=3, sigma=1.5)
    a = oracle.forward(im.points, im.values, im.H, im.W, im.sigma)["image"]
    b = oracle.forward(im.points, im.values, im.H, im.W, im.sigma, mode=oracle.TRUNCATED, k=20.0)["image"]
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)


def test_empty_point_set():
    r = oracle.forward(np.zeros((0, 2), np.float32), np.zeros((0, 3), np.float32), 4, 5, 1.0)
    assert r["image"].shape == (4, 5, 3)
    np.testing.assert_array_equal(r["image"], 0.0)
    np.testing.assert_array_equal(r["den"], 0.0)


def test_pixel_subset_matches_full():
    im = wl.tiny_random(19, 40, 15, 13, C=3, sigma=0.9)
    full = oracle.forward(im.points, im.values, im.H, im.W, im.sigma)
    pix = np.array([0, 5, 17, 100, 15 * 13 - 1])
    sub = oracle.forward(im.points, im.values, im.H, im.W, im.sigma, pixels=pix)
    np.testing.assert_array_equal(sub["image"], full["image"].reshape(-1, 3)[pix])


def test_invalid_arguments_rejected():
    p = np.zeros((1, 2), np.float32)
    v = np.zeros((1, 3), np.float32)
    with pytest.raises(ValueError):
        oracle.forward(p, v, 4, 4, 0.0)
    with pytest.raises(ValueError):
        oracle.forward(p, v, 0, 4, 1.0)


def test_pair_count_matches_kdtree():
    im = wl.tiny_random(20, 300, 32, 32, C=1, sigma=0.8, clustered=True)
    k = 6.0
    r = oracle.forward(im.points, im.values, im.H, im.W, im.sigma, k=k)
    xx, yy = _grid(im.H, im.W)
    q = np.stack([xx.ravel(), yy.ravel()], 1)
    tree = cKDTree(im.points.astype(np.float64))
    d, _ = tree.query(q)
    rad = np.sqrt(d * d + (k * im.sigma) ** 2)
    cnt = tree.query_ball_point(q, rad * (1 + 1e-12), return_length=True)
    np.testing.assert_array_equal(r["pairs"].ravel(), cnt)
    # what the radius rule drops is below the e^{-k^2/2} scale it promises
    assert r["skipped"].max() < 1e-6


# ---------------------------------------------------------------- gradients
def _loss(points, values, H, W, s, g, mode=oracle.EXACT, k=6.0):
    return float(np.sum(oracle.forward(points, values, H, W, s, mode=mode, k=k)["image"] * g))


@pytest.mark.parametrize("mode", [oracle.EXACT, oracle.TRUNCATED])
def test_gradient_finite_differences(mode):
    im, g = wl.fd_subcase(side=12, n=24)
    H, W, s = im.H, im.W, im.sigma
    k = 6.0 if mode == oracle.EXACT else 2.5
    gr = oracle.backward(im.points, im.values, H, W, s, g, mode=mode, k=k)
    h = 2.0 ** -9
    rng = np.random.default_rng(5)
    for i in rng.choice(im.N, 6, replace=False):
        for a in range(2):
            pp = im.points.copy(); pp[i, a] += h
            pm = im.points.copy(); pm[i, a] -= h
            fd = (_loss(pp, im.values, H, W, s, g, mode, k) - _loss(pm, im.values, H, W, s, g, mode, k)) / (2 * h)
            assert abs(fd - gr["points"][i, a]) <= 2e-4 * max(1.0, abs(fd)), (i, a, fd, gr["points"][i, a])
        for c in range(im.C):
            vp = im.values.copy(); vp[i, c] += h
            vm = im.values.copy(); vm[i, c] -= h
            fd = (_loss(im.points, vp, H, W, s, g, mode, k) - _loss(im.points, vm, H, W, s, g, mode, k)) / (2 * h)
            assert abs(fd - gr["values"][i, c]) <= 1e-6 * max(1.0, abs(fd)), (i, c, fd, gr["values"][i, c])
    hs = 1e-5
    fd = (_loss(im.points, im.values, H, W, s + hs, g, mode, k) - _loss(im.points, im.values, H, W, s - hs, g, mode, k)) / (2 * hs)
    assert abs(fd - gr["sigma"]) <= 1e-5 * max(1.0, abs(fd)), (fd, gr["sigma"])


def test_gradient_torch_autograd():
    torch = pytest.importorskip("torch")
    im, g = wl.fd_subcase(side=16, n=40)
    H, W = im.H, im.W
    P = torch.tensor(im.points, dtype=torch.float64, requires_grad=True)
    V = torch.tensor(im.values, dtype=torch.float64, requires_grad=True)
    S = torch.tensor(im.sigma, dtype=torch.float64, requires_grad=True)
    yy, xx = torch.meshgrid(torch.arange(H, dtype=torch.float64) + 0.5,
                            torch.arange(W, dtype=torch.float64) + 0.5, indexing="ij")
    q = torch.stack([xx.reshape(-1), yy.reshape(-1)], 1)              # [HW, 2]
    logit = -((q[:, None, :] - P[None]) ** 2).sum(-1) / (2 * S * S)   # [HW, N]
    wgt = torch.softmax(logit, dim=1)                                  # normalised densities
    img = (wgt @ V).reshape(H, W, -1)
    (img * torch.tensor(g, dtype=torch.float64)).sum().backward()
    gr = oracle.backward(im.points, im.values, H, W, im.sigma, g)
    np.testing.assert_allclose(gr["points"], P.grad.numpy(), rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(gr["values"], V.grad.numpy(), rtol=1e-9, atol=1e-11)
    assert math.isclose(gr["sigma"], float(S.grad), rel_tol=1e-9, abs_tol=1e-11)
    # the forward of the autograd version agrees with the oracle too
    np.testing.assert_allclose(img.detach().numpy(),
                               oracle.forward(im.points, im.values, H, W, im.sigma)["image"],
                               rtol=0, atol=1e-13)


def test_value_gradient_sums_to_upstream_sum():
    im, g = wl.fd_subcase(side=10, n=30)
    gr = oracle.backward(im.points, im.values, im.H, im.W, im.sigma, g)
    np.testing.assert_allclose(gr["values"].sum(0), g.reshape(-1, im.C).astype(np.float64).sum(0),
                               rtol=1e-12, atol=1e-10)
    # translating every point and every pixel together changes nothing, so the
    # position gradients of an exact evaluation sum to minus the pixel-side
    # derivative; with the pixels fixed this is sum_i dL/dmu_i = -sum_q dL/dq,
    # which for a full-frame loss is checked by moving all points at once:
    h = 2.0 ** -9
    sh = np.array([h, 0.0], np.float32)
    fd = (_loss(im.points + sh, im.values, im.H, im.W, im.sigma, g)
          - _loss(im.points - sh, im.values, im.H, im.W, im.sigma, g)) / (2 * h)
    assert abs(fd - gr["points"][:, 0].sum()) <= 2e-4 * max(1.0, abs(fd))


# ------------------------------------------------------ per-point sigma (extension)
def _pp_case(seed, n, H, W, C=3, lo=0.5, hi=2.0):
    rng = np.random.default_rng(seed)
    pts = np.stack([rng.uniform(0, W, n), rng.uniform(0, H, n)], 1).astype(np.float32)
    vals = rng.uniform(0, 1, (n, C)).astype(np.float32)
    sig = rng.uniform(lo, hi, n).astype(np.float32)
    return pts, vals, sig


@pytest.mark.parametrize("mode", [oracle.EXACT, oracle.TRUNCATED])
def test_pp_equal_sigmas_reduce_to_the_shared_oracle(mode):
    """With every sigma_i = sigma the normalisers are equal and cancel: the
    per-point evaluation is the (pinned) shared-sigma one, and the per-point
    sigma gradients sum to the shared sigma gradient (the -2/sigma terms
    cancel over the normalised weights)."""
    pts, vals, _ = _pp_case(1, 40, 13, 17)
    s = np.float32(1.3)
    sig = np.full(40, s, np.float32)
    k = 6.0 if mode == oracle.EXACT else 2.5
    a = oracle.forward_pp(pts, vals, sig, 13, 17, mode=mode, k=k)
    b = oracle.forward(pts, vals, 13, 17, float(s), mode=mode, k=k)
    np.testing.assert_allclose(a["image"], b["image"], rtol=0, atol=1e-13)
    g = np.random.default_rng(2).standard_normal((13, 17, 3)).astype(np.float32)
    ga = oracle.backward_pp(pts, vals, sig, 13, 17, g, mode=mode, k=k)
    gb = oracle.backward(pts, vals, 13, 17, float(s), g, mode=mode, k=k)
    np.testing.assert_allclose(ga["points"], gb["points"], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(ga["values"], gb["values"], rtol=1e-10, atol=1e-12)
    assert math.isclose(ga["sigmas"].sum(), gb["sigma"], rel_tol=1e-9, abs_tol=1e-11)


def test_pp_single_and_two_points():
    H, W = 9, 11
    xx, yy = _grid(H, W)
    p1 = np.float32([[3.3, 4.6]])
    c1 = np.float32([[0.2, 0.7, 0.9]])
    r = oracle.forward_pp(p1, c1, np.float32([0.8]), H, W)
    np.testing.assert_allclose(r["image"], np.broadcast_to(c1[0], (H, W, 3)), rtol=0, atol=1e-15)
    rt = oracle.forward_pp(p1, c1, np.float32([0.8]), H, W, mode=oracle.TRUNCATED, k=2.0)
    inside = (xx - float(p1[0, 0])) ** 2 + (yy - float(p1[0, 1])) ** 2 <= (2.0 * float(np.float32(0.8))) ** 2
    np.testing.assert_allclose(rt["image"][inside], np.broadcast_to(c1[0], (inside.sum(), 3)), atol=1e-15)
    assert (rt["image"][~inside] == 0).all()
    # two points with sigmas s1, s2: a logistic sigmoid of the log-weight difference
    p2 = np.float32([[2.1, 3.0], [7.4, 5.5]])
    c2 = np.float32([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    s2 = np.float32([0.9, 1.7])
    r2 = oracle.forward_pp(p2, c2, s2, H, W)
    p64 = p2.astype(np.float64)   # the oracle sees the float32 positions
    d1 = (xx - p64[0, 0]) ** 2 + (yy - p64[0, 1]) ** 2
    d2 = (xx - p64[1, 0]) ** 2 + (yy - p64[1, 1]) ** 2
    l1 = -d1 / (2 * float(s2[0]) ** 2) - 2 * math.log(float(s2[0]))
    l2 = -d2 / (2 * float(s2[1]) ** 2) - 2 * math.log(float(s2[1]))
    np.testing.assert_allclose(r2["image"][..., 1], expit(l2 - l1), rtol=0, atol=1e-12)


@pytest.mark.parametrize("mode", [oracle.EXACT, oracle.TRUNCATED])
def test_pp_torch_autograd(mode):
    """An independent FP64 torch evaluation of the per-point Eq. 1 (a softmax
    of the log-weights in exact mode, masked weights in truncated mode) and
    its autograd gradients, including each point's sigma."""
    torch = pytest.importorskip("torch")
    H, W, k = 14, 12, 2.5
    pts, vals, sig = _pp_case(7, 30, H, W)
    g = np.random.default_rng(8).standard_normal((H, W, 3)).astype(np.float32)
    P = torch.tensor(pts, dtype=torch.float64, requires_grad=True)
    V = torch.tensor(vals, dtype=torch.float64, requires_grad=True)
    S = torch.tensor(sig, dtype=torch.float64, requires_grad=True)
    yy, xx = torch.meshgrid(torch.arange(H, dtype=torch.float64) + 0.5,
                            torch.arange(W, dtype=torch.float64) + 0.5, indexing="ij")
    q = torch.stack([xx.reshape(-1), yy.reshape(-1)], 1)
    d2 = ((q[:, None, :] - P[None]) ** 2).sum(-1)
    logw = -d2 / (2 * S * S) - 2 * torch.log(S)
    if mode == oracle.EXACT:
        wgt = torch.softmax(logw, dim=1)
    else:
        w = torch.where(d2 <= (k * S) ** 2, torch.exp(logw), torch.zeros_like(d2))
        z = w.sum(1, keepdim=True)
        wgt = torch.where(z > 0, w / torch.where(z > 0, z, torch.ones_like(z)), torch.zeros_like(w))
    img = (wgt @ V).reshape(H, W, 3)
    (img * torch.tensor(g, dtype=torch.float64)).sum().backward()
    ref = oracle.forward_pp(pts, vals, sig, H, W, mode=mode, k=k)
    np.testing.assert_allclose(ref["image"], img.detach().numpy(), rtol=0, atol=1e-12)
    gr = oracle.backward_pp(pts, vals, sig, H, W, g, mode=mode, k=k)
    np.testing.assert_allclose(gr["points"], P.grad.numpy(), rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(gr["values"], V.grad.numpy(), rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(gr["sigmas"], S.grad.numpy(), rtol=1e-8, atol=1e-10)


def test_pp_sigma_gradient_finite_differences():
    H, W = 10, 12
    pts, vals, sig = _pp_case(11, 16, H, W)
    g = np.random.default_rng(12).standard_normal((H, W, 3)).astype(np.float32)

    def loss(s):
        return float((oracle.forward_pp(pts, vals, s, H, W)["image"] * g).sum())

    gr = oracle.backward_pp(pts, vals, sig, H, W, g)
    h = 2.0 ** -10
    for i in (0, 5, 11):
        sp, sm = sig.copy(), sig.copy()
        sp[i] += h
        sm[i] -= h
        fd = (loss(sp) - loss(sm)) / (float(sp[i]) - float(sm[i]))
        assert abs(fd - gr["sigmas"][i]) <= 1e-4 * max(1.0, abs(fd)), (i, fd, gr["sigmas"][i])


def test_pp_permutation_invariance():
    pts, vals, sig = _pp_case(13, 25, 8, 9)
    perm = np.random.default_rng(14).permutation(25)
    a = oracle.forward_pp(pts, vals, sig, 8, 9)["image"]
    b = oracle.forward_pp(pts[perm], vals[perm], sig[perm], 8, 9)["image"]
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)


# ------------------------------------------- anisotropic (axis-aligned) sigma (extension)
def _an_case(seed, n, H, W, C=3, lo=0.5, hi=2.0):
    pts, vals, _ = _pp_case(seed, n, H, W, C=C)
    rng = np.random.default_rng(seed + 1000)
    sxy = rng.uniform(lo, hi, (n, 2)).astype(np.float32)
    return pts, vals, sxy


@pytest.mark.parametrize("mode", [oracle.EXACT, oracle.TRUNCATED])
def test_aniso_equal_axes_reduce_to_per_point(mode):
    """sx_i = sy_i = sigma_i is the (pinned) per-point isotropic evaluation;
    the two axis gradients of a point sum to its sigma gradient."""
    pts, vals, sig = _pp_case(21, 35, 12, 15)
    sxy = np.stack([sig, sig], 1)
    k = 6.0 if mode == oracle.EXACT else 2.5
    a = oracle.forward_aniso(pts, vals, sxy, 12, 15, mode=mode, k=k)
    b = oracle.forward_pp(pts, vals, sig, 12, 15, mode=mode, k=k)
    for key in ("image", "den", "shift"):
        np.testing.assert_allclose(a[key], b[key], rtol=1e-13, atol=1e-13)
    assert (a["pairs"] == b["pairs"]).all()
    g = np.random.default_rng(22).standard_normal((12, 15, 3)).astype(np.float32)
    ga = oracle.backward_aniso(pts, vals, sxy, 12, 15, g, mode=mode, k=k)
    gb = oracle.backward_pp(pts, vals, sig, 12, 15, g, mode=mode, k=k)
    np.testing.assert_allclose(ga["points"], gb["points"], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(ga["values"], gb["values"], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(ga["sigmas_xy"].sum(1), gb["sigmas"], rtol=1e-10, atol=1e-12)


def test_aniso_single_and_two_points():
    H, W = 10, 13
    xx, yy = _grid(H, W)
    p1 = np.float32([[5.3, 4.1]])
    c1 = np.float32([[0.3, 0.6, 0.1]])
    s1 = np.float32([[2.2, 0.7]])
    sx, sy = float(s1[0, 0]), float(s1[0, 1])
    dx, dy = xx - float(p1[0, 0]), yy - float(p1[0, 1])
    r = oracle.forward_aniso(p1, c1, s1, H, W, mode=oracle.TRUNCATED, k=2.0)
    maha = dx * dx / (sx * sx) + dy * dy / (sy * sy)
    inside = maha <= 4.0
    assert inside.sum() > 3 and (~inside).sum() > 3
    np.testing.assert_allclose(r["image"][inside], np.broadcast_to(c1[0], (inside.sum(), 3)), atol=1e-15)
    assert (r["image"][~inside] == 0).all()
    # den is the 2D normal's density (times 2 pi): exp(-maha/2) / (sx sy)
    np.testing.assert_allclose(r["den"][inside], np.exp(-0.5 * maha[inside]) / (sx * sy), rtol=1e-13)
    # two points: a logistic sigmoid of the log-weight difference
    p2 = np.float32([[2.5, 3.2], [9.1, 6.4]])
    c2 = np.float32([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    s2 = np.float32([[0.8, 1.9], [2.4, 1.1]])
    r2 = oracle.forward_aniso(p2, c2, s2, H, W)
    p64, s64 = p2.astype(np.float64), s2.astype(np.float64)

    def logw(i):
        ex, ey = xx - p64[i, 0], yy - p64[i, 1]
        return -0.5 * (ex * ex / s64[i, 0] ** 2 + ey * ey / s64[i, 1] ** 2) - math.log(s64[i, 0] * s64[i, 1])

    np.testing.assert_allclose(r2["image"][..., 1], expit(logw(1) - logw(0)), rtol=0, atol=1e-12)


@pytest.mark.parametrize("mode", [oracle.EXACT, oracle.TRUNCATED])
def test_aniso_axis_swap_transposes(mode):
    """Swapping x and y in the points and the sigmas, and H with W, transposes
    the image and swaps the gradients' axes."""
    H, W = 11, 8
    pts, vals, sxy = _an_case(23, 30, H, W)
    k = 6.0 if mode == oracle.EXACT else 2.0
    a = oracle.forward_aniso(pts, vals, sxy, H, W, mode=mode, k=k)
    b = oracle.forward_aniso(pts[:, ::-1].copy(), vals, sxy[:, ::-1].copy(), W, H, mode=mode, k=k)
    np.testing.assert_allclose(b["image"], a["image"].transpose(1, 0, 2), rtol=0, atol=1e-13)
    g = np.random.default_rng(24).standard_normal((H, W, 3)).astype(np.float32)
    ga = oracle.backward_aniso(pts, vals, sxy, H, W, g, mode=mode, k=k)
    gb = oracle.backward_aniso(pts[:, ::-1].copy(), vals, sxy[:, ::-1].copy(), W, H,
                               g.transpose(1, 0, 2).copy(), mode=mode, k=k)
    np.testing.assert_allclose(gb["points"], ga["points"][:, ::-1], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(gb["sigmas_xy"], ga["sigmas_xy"][:, ::-1], rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("mode", [oracle.EXACT, oracle.TRUNCATED])
def test_aniso_torch_autograd(mode):
    """An independent FP64 torch evaluation (softmax of the anisotropic
    log-weights, or masked weights inside the ellipses) and its autograd
    gradients, including both axes of every point's sigma."""
    torch = pytest.importorskip("torch")
    H, W, k = 13, 14, 2.5
    pts, vals, sxy = _an_case(25, 28, H, W)
    g = np.random.default_rng(26).standard_normal((H, W, 3)).astype(np.float32)
    P = torch.tensor(pts, dtype=torch.float64, requires_grad=True)
    V = torch.tensor(vals, dtype=torch.float64, requires_grad=True)
    S = torch.tensor(sxy, dtype=torch.float64, requires_grad=True)
    yy, xx = torch.meshgrid(torch.arange(H, dtype=torch.float64) + 0.5,
                            torch.arange(W, dtype=torch.float64) + 0.5, indexing="ij")
    q = torch.stack([xx.reshape(-1), yy.reshape(-1)], 1)
    e = (q[:, None, :] - P[None]) / S[None]
    m2 = (e * e).sum(-1)
    logw = -0.5 * m2 - torch.log(S[:, 0] * S[:, 1])
    if mode == oracle.EXACT:
        wgt = torch.softmax(logw, dim=1)
    else:
        w = torch.where(m2 <= k * k, torch.exp(logw), torch.zeros_like(m2))
        z = w.sum(1, keepdim=True)
        wgt = torch.where(z > 0, w / torch.where(z > 0, z, torch.ones_like(z)), torch.zeros_like(w))
    img = (wgt @ V).reshape(H, W, 3)
    (img * torch.tensor(g, dtype=torch.float64)).sum().backward()
    ref = oracle.forward_aniso(pts, vals, sxy, H, W, mode=mode, k=k)
    np.testing.assert_allclose(ref["image"], img.detach().numpy(), rtol=0, atol=1e-12)
    gr = oracle.backward_aniso(pts, vals, sxy, H, W, g, mode=mode, k=k)
    np.testing.assert_allclose(gr["points"], P.grad.numpy(), rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(gr["values"], V.grad.numpy(), rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(gr["sigmas_xy"], S.grad.numpy(), rtol=1e-8, atol=1e-10)


def test_aniso_sigma_gradient_finite_differences():
    H, W = 10, 11
    pts, vals, sxy = _an_case(27, 14, H, W)
    g = np.random.default_rng(28).standard_normal((H, W, 3)).astype(np.float32)

    def loss(s):
        return float((oracle.forward_aniso(pts, vals, s, H, W)["image"] * g).sum())

    gr = oracle.backward_aniso(pts, vals, sxy, H, W, g)
    h = 2.0 ** -10
    for i, ax in ((0, 0), (4, 1), (9, 0), (13, 1)):
        sp, sm = sxy.copy(), sxy.copy()
        sp[i, ax] += h
        sm[i, ax] -= h
        fd = (loss(sp) - loss(sm)) / (float(sp[i, ax]) - float(sm[i, ax]))
        assert abs(fd - gr["sigmas_xy"][i, ax]) <= 1e-4 * max(1.0, abs(fd)), (i, ax, fd, gr["sigmas_xy"][i, ax])


def test_aniso_permutation_invariance():
    pts, vals, sxy = _an_case(29, 25, 8, 9)
    perm = np.random.default_rng(30).permutation(25)
    a = oracle.forward_aniso(pts, vals, sxy, 8, 9)["image"]
    b = oracle.forward_aniso(pts[perm], vals[perm], sxy[perm], 8, 9)["image"]
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)


# --------------------------------------------------- full covariance per point (extension)
def _cov_case(seed, n, H, W, C=3, lo=0.6, hi=2.0, rmax=0.8):
    pts, vals, _ = _pp_case(seed, n, H, W, C=C)
    rng = np.random.default_rng(seed + 2000)
    cov = np.concatenate([rng.uniform(lo, hi, (n, 2)), rng.uniform(-rmax, rmax, (n, 1))], 1).astype(np.float32)
    return pts, vals, cov


def _cov_matrix(c):
    sx, sy, r = (float(v) for v in c)
    return np.array([[sx * sx, r * sx * sy], [r * sx * sy, sy * sy]])


@pytest.mark.parametrize("mode", [oracle.EXACT, oracle.TRUNCATED])
def test_cov_zero_correlation_reduces_to_aniso(mode):
    pts, vals, cov = _cov_case(41, 30, 12, 14)
    cov[:, 2] = 0.0
    k = 6.0 if mode == oracle.EXACT else 2.5
    a = oracle.forward_cov(pts, vals, cov, 12, 14, mode=mode, k=k)
    b = oracle.forward_aniso(pts, vals, cov[:, :2].copy(), 12, 14, mode=mode, k=k)
    for key in ("image", "den", "shift"):
        np.testing.assert_allclose(a[key], b[key], rtol=1e-13, atol=1e-13)
    assert (a["pairs"] == b["pairs"]).all()
    g = np.random.default_rng(42).standard_normal((12, 14, 3)).astype(np.float32)
    ga = oracle.backward_cov(pts, vals, cov, 12, 14, g, mode=mode, k=k)
    gb = oracle.backward_aniso(pts, vals, cov[:, :2].copy(), 12, 14, g, mode=mode, k=k)
    np.testing.assert_allclose(ga["points"], gb["points"], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(ga["values"], gb["values"], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(ga["cov"][:, :2], gb["sigmas_xy"], rtol=1e-10, atol=1e-12)


def test_cov_single_point_ellipse_and_density():
    """One point: colour inside the rotated ellipse d^T S^-1 d <= k^2 and 0
    outside; den = exp(-Q/2) / sqrt(det S), with S^-1 and det S taken by
    numpy's matrix routines."""
    H, W, k = 12, 13, 2.0
    xx, yy = _grid(H, W)
    p1 = np.float32([[6.2, 5.7]])
    c1 = np.float32([[0.4, 0.1, 0.8]])
    cv = np.float32([[2.3, 1.1, 0.65]])
    r = oracle.forward_cov(p1, c1, cv, H, W, mode=oracle.TRUNCATED, k=k)
    S = _cov_matrix(cv[0])
    Si = np.linalg.inv(S)
    d = np.stack([xx - float(p1[0, 0]), yy - float(p1[0, 1])], -1)
    Q = np.einsum("...i,ij,...j->...", d, Si, d)
    inside = Q <= k * k
    assert inside.sum() > 5 and (~inside).sum() > 5
    np.testing.assert_allclose(r["image"][inside], np.broadcast_to(c1[0], (inside.sum(), 3)), atol=1e-15)
    assert (r["image"][~inside] == 0).all()
    np.testing.assert_allclose(r["den"][inside], np.exp(-0.5 * Q[inside]) / math.sqrt(np.linalg.det(S)),
                               rtol=1e-12)


@pytest.mark.parametrize("mode", [oracle.EXACT, oracle.TRUNCATED])
def test_cov_symmetries(mode):
    """Transposing the problem (x <-> y, sx <-> sy, H <-> W) transposes the
    image; mirroring x (x -> W - x, rho -> -rho) mirrors the columns; the
    gradients follow (the mirrored x and rho gradients change sign)."""
    H, W = 10, 9
    pts, vals, cov = _cov_case(43, 28, H, W)
    pts = (np.round(pts * 1024.0) / 1024.0).astype(np.float32)   # W - x stays exact in float32
    k = 6.0 if mode == oracle.EXACT else 2.0
    g = np.random.default_rng(44).standard_normal((H, W, 3)).astype(np.float32)
    a = oracle.forward_cov(pts, vals, cov, H, W, mode=mode, k=k)
    ga = oracle.backward_cov(pts, vals, cov, H, W, g, mode=mode, k=k)
    tc = cov[:, [1, 0, 2]].copy()
    b = oracle.forward_cov(pts[:, ::-1].copy(), vals, tc, W, H, mode=mode, k=k)
    np.testing.assert_allclose(b["image"], a["image"].transpose(1, 0, 2), rtol=0, atol=1e-13)
    gb = oracle.backward_cov(pts[:, ::-1].copy(), vals, tc, W, H, g.transpose(1, 0, 2).copy(), mode=mode, k=k)
    np.testing.assert_allclose(gb["points"], ga["points"][:, ::-1], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(gb["cov"], ga["cov"][:, [1, 0, 2]], rtol=1e-10, atol=1e-12)
    mp = pts.copy()
    mp[:, 0] = np.float32(W) - mp[:, 0]
    mc = cov.copy()
    mc[:, 2] = -mc[:, 2]
    m = oracle.forward_cov(mp, vals, mc, H, W, mode=mode, k=k)
    np.testing.assert_allclose(m["image"], a["image"][:, ::-1], rtol=0, atol=1e-13)
    gm = oracle.backward_cov(mp, vals, mc, H, W, g[:, ::-1].copy(), mode=mode, k=k)
    np.testing.assert_allclose(gm["points"], ga["points"] * np.array([-1.0, 1.0]), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(gm["cov"], ga["cov"] * np.array([1.0, 1.0, -1.0]), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("mode", [oracle.EXACT, oracle.TRUNCATED])
def test_cov_torch_autograd(mode):
    """An independent FP64 torch evaluation built from the covariance matrix
    (torch.linalg.inv, torch.logdet) and its autograd gradients with respect
    to positions, values and (sx, sy, rho)."""
    torch = pytest.importorskip("torch")
    H, W, k = 12, 13, 2.5
    pts, vals, cov = _cov_case(45, 26, H, W)
    g = np.random.default_rng(46).standard_normal((H, W, 3)).astype(np.float32)
    P = torch.tensor(pts, dtype=torch.float64, requires_grad=True)
    V = torch.tensor(vals, dtype=torch.float64, requires_grad=True)
    CV = torch.tensor(cov, dtype=torch.float64, requires_grad=True)
    sx, sy, r = CV[:, 0], CV[:, 1], CV[:, 2]
    S = torch.stack([torch.stack([sx * sx, r * sx * sy], -1), torch.stack([r * sx * sy, sy * sy], -1)], -2)
    Si = torch.linalg.inv(S)
    yy, xx = torch.meshgrid(torch.arange(H, dtype=torch.float64) + 0.5,
                            torch.arange(W, dtype=torch.float64) + 0.5, indexing="ij")
    q = torch.stack([xx.reshape(-1), yy.reshape(-1)], 1)
    d = q[:, None, :] - P[None]
    Q = torch.einsum("pni,nij,pnj->pn", d, Si, d)
    logw = -0.5 * Q - 0.5 * torch.logdet(S)
    if mode == oracle.EXACT:
        wgt = torch.softmax(logw, dim=1)
    else:
        w = torch.where(Q <= k * k, torch.exp(logw), torch.zeros_like(Q))
        z = w.sum(1, keepdim=True)
        wgt = torch.where(z > 0, w / torch.where(z > 0, z, torch.ones_like(z)), torch.zeros_like(w))
    img = (wgt @ V).reshape(H, W, 3)
    (img * torch.tensor(g, dtype=torch.float64)).sum().backward()
    ref = oracle.forward_cov(pts, vals, cov, H, W, mode=mode, k=k)
    np.testing.assert_allclose(ref["image"], img.detach().numpy(), rtol=0, atol=1e-12)
    gr = oracle.backward_cov(pts, vals, cov, H, W, g, mode=mode, k=k)
    np.testing.assert_allclose(gr["points"], P.grad.numpy(), rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(gr["values"], V.grad.numpy(), rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(gr["cov"], CV.grad.numpy(), rtol=1e-8, atol=1e-10)


def test_cov_gradient_finite_differences():
    H, W = 10, 11
    pts, vals, cov = _cov_case(47, 14, H, W)
    g = np.random.default_rng(48).standard_normal((H, W, 3)).astype(np.float32)

    def loss(c):
        return float((oracle.forward_cov(pts, vals, c, H, W)["image"] * g).sum())

    gr = oracle.backward_cov(pts, vals, cov, H, W, g)
    h = 2.0 ** -10
    for i, ax in ((0, 0), (3, 1), (6, 2), (11, 2), (13, 0)):
        cp, cm = cov.copy(), cov.copy()
        cp[i, ax] += h
        cm[i, ax] -= h
        fd = (loss(cp) - loss(cm)) / (float(cp[i, ax]) - float(cm[i, ax]))
        assert abs(fd - gr["cov"][i, ax]) <= 1e-4 * max(1.0, abs(fd)), (i, ax, fd, gr["cov"][i, ax])


def test_cov_permutation_invariance_and_rejects_degenerate():
    pts, vals, cov = _cov_case(49, 25, 8, 9)
    perm = np.random.default_rng(50).permutation(25)
    a = oracle.forward_cov(pts, vals, cov, 8, 9)["image"]
    b = oracle.forward_cov(pts[perm], vals[perm], cov[perm], 8, 9)["image"]
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)
    bad = cov.copy()
    bad[3, 2] = 1.0
    with pytest.raises(ValueError):
        oracle.forward_cov(pts, vals, bad, 8, 9)
