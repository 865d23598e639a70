"""Exact mode with a sigma (axis-aligned pair, full covariance) per point:
Eq. 1 over all points with each point its own normal N(mu_i, S_i), its
normaliser kept.  The CUDA path against the FP64 oracle's forward_pp /
forward_aniso / forward_cov and their backward passes in exact mode.

Bars: forward max-abs <= 1e-4 on colours in [0, 1] at every pixel (nothing is
masked: in exact mode every point counts everywhere); den (the weights' sum
relative to the pixel's largest weight) relative 1e-4; gradients per tensor
max|g_gpu - g_ref| <= 1e-3 max|g_ref|, and element by element relative 1e-3
wherever |g_ref| >= 1% of the tensor's largest.  k = 6 throughout: points
below exp(-18) of a pixel's largest weight may be left out, far below the
forward bar."""
import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_helpers import TOL_FWD, sample_pixels, to_dev

pytestmark = pytest.mark.gpu

TOL_BWD = 1e-3
REL_FLOOR = 1e-2
K = 6.0


def gmi():
    import paper_2012_13257_b300 as g
    return g


ORACLE_FWD = {1: oracle.forward_pp, 2: oracle.forward_aniso, 3: oracle.forward_cov}
ORACLE_BWD = {1: oracle.backward_pp, 2: oracle.backward_aniso, 3: oracle.backward_cov}
GRAD_KEY = {1: "sigmas", 2: "sigmas_xy", 3: "cov"}


def draw_sigmas(kind, seed, N, lo, hi):
    """Per-point sigmas of the given kind and the bound the call takes."""
    if kind == 1:
        s = wl.point_sigmas(seed, N, lo, hi)
        return s, float(s.max()) if N else hi
    if kind == 2:
        s = wl.point_sigmas(seed, N, lo, hi, axes=2)
        return s, float(s.max()) if N else hi
    s = wl.point_cov(seed, N, lo, hi, rmax=0.9)
    return s, wl.cov_bound(s)


def corner_points(im, frac):
    """The image's points squeezed into the top-left frac x frac of the frame,
    so that most pixels lie far from every point (the far field)."""
    pts = im.points.astype(np.float64) * frac
    return wl.Image(pts.astype(np.float32), im.values, im.sigma, im.H, im.W)


def run(im, sig, bound, dev, **kw):
    import torch
    img, den = gmi().interpolate_pp(to_dev(im.points, dev), to_dev(im.values, dev), to_dev(sig, dev), bound,
                                    im.H, im.W, radius_sigmas=K, mode="exact", return_aux=True, check=True, **kw)
    torch.cuda.synchronize()
    return img.cpu().numpy(), den.cpu().numpy()


def check_forward(kind, im, sig, bound, dev, **kw):
    out, den = run(im, sig, bound, dev, **kw)
    ref = ORACLE_FWD[kind](im.points, im.values, sig, im.H, im.W, mode=oracle.EXACT, k=K)
    assert np.isfinite(out).all() and np.isfinite(den).all()
    err = np.abs(out.astype(np.float64) - ref["image"]).max()
    assert err <= TOL_FWD, err
    rel = (np.abs(den.astype(np.float64) - ref["den"]) / ref["den"]).max()
    assert rel <= 1e-4, rel
    assert (den >= 1.0 - 1e-4).all()   # the largest weight counts 1 (up to rounding)
    return out, ref


CASES = [  # (seed, N, H, W, C, sigma lo, sigma hi, layout)
    (1, 300, 37, 53, 3, 0.5, 1.5, "uniform"),
    (2, 800, 64, 96, 1, 0.3, 2.0, "clustered"),
    (3, 500, 45, 61, 4, 0.05, 1.2, "clustered"),
    (4, 200, 29, 31, 2, 1.0, 3.0, "margin"),
    (5, 400, 70, 83, 3, 0.4, 0.9, "corner"),
    (6, 60, 66, 90, 3, 0.5, 1.5, "corner"),
]


def make_case(case, kind):
    seed, N, H, W, C, lo, hi, layout = case
    im = wl.tiny_random(seed, N, H, W, C=C, sigma=hi, clustered=layout in ("clustered", "corner"),
                        margin=4.0 if layout == "margin" else 0.0)
    if layout == "corner":
        im = corner_points(im, 0.25)
    sig, bound = draw_sigmas(kind, seed + 7 * kind, N, lo, hi)
    return im, sig, bound


def ids(c):
    return "s%d_N%d_%dx%d_C%d_%s" % (c[:5] + (c[7],))


@pytest.mark.parametrize("case", CASES, ids=ids)
@pytest.mark.parametrize("kind", [1, 2, 3], ids=["iso", "aniso", "cov"])
def test_forward_matches_oracle(cuda_device, case, kind):
    im, sig, bound = make_case(case, kind)
    check_forward(kind, im, sig, bound, cuda_device)


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("kind", [1, 3], ids=["iso", "cov"])
def test_forward_variants(cuda_device, variant, kind):
    im, sig, bound = make_case(CASES[2], kind)
    check_forward(kind, im, sig, bound, cuda_device, variant=variant)


def test_far_pixels_blend_nearest_points(cuda_device):
    """Two points in one corner of a 96^2 frame: a pixel 100 px away still
    gets their weighted blend (truncated mode would give 0 there), and it
    matches the oracle."""
    pts = np.float32([[3.2, 4.1], [5.7, 2.9]])
    vals = np.float32([[1.0, 0.0, 0.25], [0.0, 1.0, 0.75]])
    sig = np.float32([0.6, 0.9])
    im = wl.Image(pts, vals, 0.9, 96, 96)
    out, _ = run(im, sig, 0.9, cuda_device)
    ref = oracle.forward_pp(pts, vals, sig, 96, 96, mode=oracle.EXACT, k=K)
    assert np.abs(out - ref["image"]).max() <= TOL_FWD
    far = out[95, 95]
    assert far.sum() > 0.99 and abs(far[0] + far[1] - 1.0) <= 1e-5


def test_single_point_and_empty(cuda_device):
    """One point: every pixel takes its colour (Eq. 1 with one term); no
    point: zeros."""
    im = wl.Image(np.float32([[10.3, 7.8]]), np.float32([[0.2, 0.4, 0.9]]), 1.0, 41, 57)
    for kind, sig in ((1, np.float32([0.7])), (2, np.float32([[0.7, 0.4]])), (3, np.float32([[0.7, 0.4, 0.5]]))):
        bound = wl.cov_bound(sig) if kind == 3 else 0.7
        out, den = run(im, sig, bound, cuda_device)
        np.testing.assert_allclose(out, np.broadcast_to(im.values[0], out.shape), rtol=0, atol=1e-6)
        np.testing.assert_allclose(den, 1.0, rtol=0, atol=1e-5)
    empty = wl.Image(np.zeros((0, 2), np.float32), np.zeros((0, 3), np.float32), 1.0, 19, 23)
    out, den = run(empty, np.zeros(0, np.float32), 1.0, cuda_device)
    assert (out == 0).all() and (den == 0).all()


def test_equal_sigmas_match_shared_exact(cuda_device):
    """With every sigma_i = sigma the normalisers are equal and cancel: the
    shared-sigma exact forward's image."""
    import torch
    im = wl.tiny_random(13, 700, 50, 66, C=3, sigma=0.8, clustered=True)
    sig = np.full(im.N, im.sigma, np.float32)
    a, da = run(im, sig, im.sigma, cuda_device)
    P, V = to_dev(im.points, cuda_device), to_dev(im.values, cuda_device)
    b = gmi().interpolate(P, V, im.sigma, im.H, im.W, mode="exact", radius_sigmas=K)
    torch.cuda.synchronize()
    assert np.abs(a - b.cpu().numpy()).max() <= 1e-5


def test_loose_bound_same_result(cuda_device):
    """The bound sets only the search radius and the reference scale of the
    normalisers, which cancel: a loose one gives the same image."""
    im, sig, bound = make_case(CASES[1], 1)
    a, da = run(im, sig, bound, cuda_device)
    b, db = run(im, sig, 2.5 * bound, cuda_device)
    assert np.abs(a - b).max() <= 1e-5
    np.testing.assert_allclose(da, db, rtol=1e-5)


def test_graph_replay(cuda_device):
    import torch
    g = gmi()
    im, sig, bound = make_case(CASES[0], 1)
    P, V, S = to_dev(im.points, cuda_device), to_dev(im.values, cuda_device), to_dev(sig, cuda_device)
    want = g.interpolate_pp(P, V, S, bound, im.H, im.W, mode="exact").cpu().numpy()
    out = torch.empty((im.H, im.W, 3), dtype=torch.float32, device=cuda_device)
    for _ in range(3):
        out.zero_()
        g.interpolate_pp(P, V, S, bound, im.H, im.W, mode="exact", graph=True, out=out)
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), want, rtol=0, atol=1e-6)


def test_full_size_sampled(cuda_device):
    """The 512^2 -> 1024^2 upsampling workload with sigma_i log-uniform in
    [0.5, 1.5] px, exact mode, on a pixel sample that includes the pixels
    farthest from any point."""
    im = wl.upsample_1024()
    sig = wl.point_sigmas(17, im.N, 0.5, 1.5)
    out, den = run(im, sig, 1.5, cuda_device)
    pix = sample_pixels(im.points, im.H, im.W)
    ref = oracle.forward_pp(im.points, im.values, sig, im.H, im.W, mode=oracle.EXACT, k=K, pixels=pix)
    assert np.abs(out.reshape(-1, 3)[pix] - ref["image"]).max() <= TOL_FWD
    rel = np.abs(den.reshape(-1)[pix].astype(np.float64) - ref["den"]) / ref["den"]
    assert rel.max() <= 1e-4


def test_cov_full_size_clustered_sampled(cuda_device):
    """A clustered 512^2 frame (wide empty regions) with full covariances,
    exact mode, on a pixel sample with its far field."""
    rng = np.random.default_rng(41)
    pts = wl.clustered_points(rng, 20000, 512, 512)
    vals = rng.uniform(0, 1, (20000, 3)).astype(np.float32)
    im = wl.Image(pts, vals, 1.5, 512, 512)
    cov = wl.point_cov(42, im.N, 0.4, 1.5, rmax=0.9)
    out, den = run(im, cov, wl.cov_bound(cov), cuda_device)
    pix = sample_pixels(im.points, im.H, im.W, n_random=1024)
    ref = oracle.forward_cov(im.points, im.values, cov, im.H, im.W, mode=oracle.EXACT, k=K, pixels=pix)
    assert np.abs(out.reshape(-1, 3)[pix] - ref["image"]).max() <= TOL_FWD


# ------------------------------------------------------------------ backward
def gpu_grads(im, sig, bound, g_up, dev, **kw):
    import torch
    G = gmi()
    P, V, S = to_dev(im.points, dev), to_dev(im.values, dev), to_dev(sig, dev)
    img, den = G.interpolate_pp(P, V, S, bound, im.H, im.W, radius_sigmas=K, mode="exact", return_aux=True, **kw)
    gp, gv, gs = G.interpolate_backward_pp(P, V, S, bound, im.H, im.W, img, den, to_dev(g_up, dev),
                                           radius_sigmas=K, mode="exact", check=True, **kw)
    torch.cuda.synchronize()
    return gp.cpu().numpy(), gv.cpu().numpy(), gs.cpu().numpy()


def assert_grads(got, ref, kind, tol=TOL_BWD):
    """Per tensor: max |g - g_ref| <= tol max |g_ref|, and element by element
    |g - g_ref| <= tol |g_ref| wherever |g_ref| >= REL_FLOOR max |g_ref|."""
    for name, a, b in zip(("points", "values", GRAD_KEY[kind]), got,
                          (ref["points"], ref["values"], ref[GRAD_KEY[kind]])):
        b = np.asarray(b).reshape(a.shape)
        scale = np.abs(b).max()
        diff = np.abs(a.astype(np.float64) - b)
        assert np.isfinite(a).all(), name
        assert diff.max() <= tol * max(scale, 1e-30), "%s: max err %.3g vs scale %.3g" % (name, diff.max(), scale)
        big = np.abs(b) >= REL_FLOOR * scale
        rel = (diff[big] / np.abs(b[big])).max() if big.any() else 0.0
        assert rel <= tol, "%s: element-wise relative err %.3g above the %.0e floor" % (name, rel, REL_FLOOR)


@pytest.mark.parametrize("case", CASES, ids=ids)
@pytest.mark.parametrize("kind", [1, 2, 3], ids=["iso", "aniso", "cov"])
def test_backward_matches_oracle(cuda_device, case, kind):
    im, sig, bound = make_case(case, kind)
    g = np.random.default_rng(case[0] + 100).standard_normal((im.H, im.W, im.values.shape[1])).astype(np.float32)
    ref = ORACLE_BWD[kind](im.points, im.values, sig, im.H, im.W, g, mode=oracle.EXACT, k=K)
    assert_grads(gpu_grads(im, sig, bound, g, cuda_device), ref, kind)


@pytest.mark.parametrize("variant", [1, 3])
def test_backward_variants(cuda_device, variant):
    im, sig, bound = make_case(CASES[1], 3)
    g = np.random.default_rng(7).standard_normal((im.H, im.W, im.values.shape[1])).astype(np.float32)
    ref = oracle.backward_cov(im.points, im.values, sig, im.H, im.W, g, mode=oracle.EXACT, k=K)
    assert_grads(gpu_grads(im, sig, bound, g, cuda_device, variant=variant), ref, 3)


def test_backward_central_differences(cuda_device):
    """The CUDA gradient of a 24x24 full-covariance case against FP64 central
    differences of the oracle's exact forward on a few entries of each
    tensor.  The oracle reads float32 inputs, so the step is h = 2^-13
    (about 1.2e-4), which float32 represents exactly at these magnitudes."""
    im, sig, bound = make_case((8, 40, 24, 24, 3, 0.6, 1.8, "uniform"), 3)
    g = np.random.default_rng(8).standard_normal((24, 24, 3))
    got = gpu_grads(im, sig, bound, g.astype(np.float32), cuda_device)

    def loss(pts, vals, cov):
        r = oracle.forward_cov(pts, vals, cov, 24, 24, mode=oracle.EXACT, k=K)
        return float((r["image"].reshape(24, 24, 3) * g).sum())

    h = 2.0 ** -13
    rng = np.random.default_rng(9)
    for which, arr in ((0, im.points), (1, im.values), (2, sig)):
        for _ in range(4):
            i = int(rng.integers(0, arr.shape[0]))
            j = int(rng.integers(0, arr.shape[1]))
            args = [im.points.astype(np.float64), im.values.astype(np.float64), sig.astype(np.float64)]
            plus = [a.copy() for a in args]
            minus = [a.copy() for a in args]
            plus[which][i, j] += h
            minus[which][i, j] -= h
            assert np.float32(plus[which][i, j]) - np.float32(minus[which][i, j]) == np.float32(2 * h)
            fd = (loss(*plus) - loss(*minus)) / (2 * h)
            scale = np.abs(got[which]).max()
            assert abs(got[which][i, j] - fd) <= 2e-3 * scale + 1e-6, (which, i, j, got[which][i, j], fd)


def test_autograd_op(cuda_device):
    G = gmi()
    im, sig, bound = make_case(CASES[4], 2)
    g = np.random.default_rng(104).standard_normal((im.H, im.W, 3)).astype(np.float32)
    P = to_dev(im.points, cuda_device).requires_grad_(True)
    V = to_dev(im.values, cuda_device).requires_grad_(True)
    S = to_dev(sig, cuda_device).requires_grad_(True)
    img = G.gmi_interpolate_pp(P, V, S, bound, im.H, im.W, radius_sigmas=K)   # exact mode by default
    (img * to_dev(g, cuda_device)).sum().backward()
    ref = oracle.backward_aniso(im.points, im.values, sig, im.H, im.W, g, mode=oracle.EXACT, k=K)
    assert_grads((P.grad.cpu().numpy(), V.grad.cpu().numpy(), S.grad.cpu().numpy()), ref, 2)
