"""Per-point sigma (each point its own N(mu_i, sigma_i^2 I), normalisers
kept), truncated mode (each point counts within k sigma_i; exact mode is
covered by test_pp_exact_gpu.py): the CUDA path against the FP64 oracle's
forward_pp / backward_pp.

Bars as for the shared-sigma tests: forward max-abs <= 1e-4 on colours in
[0, 1] over pixels whose result no point on its radius decides; den relative
1e-4 (the CUDA den is the oracle's times sigma_bound^2); gradients per tensor
max|g_gpu - g_ref| <= 1e-3 max|g_ref|."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_helpers import TOL_FWD, sample_pixels, to_dev

pytestmark = pytest.mark.gpu

TOL_BWD = 1e-3


def gmi():
    import paper_2012_13257_b300 as g
    return g


def run(im, sig, bound, dev, k=6.0, **kw):
    import torch
    img, den = gmi().interpolate_pp(to_dev(im.points, dev), to_dev(im.values, dev), to_dev(sig, dev), bound,
                                    im.H, im.W, radius_sigmas=k, return_aux=True, check=True, **kw, mode="truncated")
    torch.cuda.synchronize()
    return img.cpu().numpy(), den.cpu().numpy()


def check_forward(im, sig, bound, dev, k, **kw):
    out, den = run(im, sig, bound, dev, k=k, **kw)
    ref = oracle.forward_pp(im.points, im.values, sig, im.H, im.W, mode=oracle.TRUNCATED, k=k)
    decided = ref["skipped"] < 1e-3
    assert decided.mean() > 0.99
    err = np.abs(out.astype(np.float64) - ref["image"])[decided]
    assert np.isfinite(out).all()
    assert err.max() <= TOL_FWD, err.max()
    scaled = ref["den"] * float(bound) ** 2
    live = decided & (scaled > 0)
    rel = np.abs(den.astype(np.float64) - scaled)[live] / scaled[live]
    assert rel.max() <= 1e-4, rel.max()
    empty = (ref["den"] == 0) & decided
    assert (out[empty] == 0).all() and (den[empty] == 0).all()
    return out, ref


CASES = [  # (seed, N, H, W, C, sigma lo, sigma hi, k, clustered)
    (1, 300, 37, 53, 3, 0.5, 1.5, 3.0, False),
    (2, 800, 64, 96, 1, 0.3, 2.0, 3.0, True),
    (3, 500, 45, 61, 4, 0.05, 1.2, 4.0, True),
    (4, 200, 29, 31, 2, 1.0, 3.0, 2.0, False),
    (5, 1500, 70, 83, 3, 0.4, 0.9, 6.0, True),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "s%d_N%d_%dx%d_C%d" % c[:5])
@pytest.mark.parametrize("variant", [1, 2, 3])
def test_forward_matches_oracle(cuda_device, case, variant):
    seed, N, H, W, C, lo, hi, k, clustered = case
    im = wl.tiny_random(seed, N, H, W, C=C, sigma=hi, clustered=clustered, margin=2.0 if not clustered else 0.0)
    sig = wl.point_sigmas(seed + 7, N, lo, hi)
    check_forward(im, sig, hi, cuda_device, k, variant=variant)


def test_loose_bound_same_result(cuda_device):
    """The bound only sets the search window: a loose one gives the same image."""
    im = wl.tiny_random(11, 600, 48, 52, C=3, sigma=1.0, clustered=True)
    sig = wl.point_sigmas(12, 600, 0.3, 1.0)
    a, da = run(im, sig, 1.0, cuda_device, k=3.0)
    b, db = run(im, sig, 2.5, cuda_device, k=3.0)
    assert np.abs(a - b).max() <= 2e-6
    np.testing.assert_allclose(db, da * 2.5 ** 2, rtol=2e-6, atol=0)


def test_equal_sigmas_match_shared_truncated(cuda_device):
    """With every sigma_i = sigma, the shared-sigma truncated forward (same den)."""
    import torch
    im = wl.tiny_random(13, 700, 50, 66, C=3, sigma=0.8, clustered=True)
    sig = np.full(im.N, im.sigma, np.float32)
    a, da = run(im, sig, im.sigma, cuda_device, k=3.0)
    P, V = to_dev(im.points, cuda_device), to_dev(im.values, cuda_device)
    b, db, _ = gmi().interpolate(P, V, im.sigma, im.H, im.W, mode="truncated", radius_sigmas=3.0, return_aux=True)
    torch.cuda.synchronize()
    ref = oracle.forward(im.points, im.values, im.H, im.W, im.sigma, mode=oracle.TRUNCATED, k=3.0)
    decided = ref["skipped"] < 1e-3
    assert np.abs(a - b.cpu().numpy())[decided].max() <= 1e-5
    np.testing.assert_allclose(da[decided], db.cpu().numpy()[decided], rtol=1e-5, atol=1e-30)


def test_empty_and_single_point(cuda_device):
    im = wl.Image(np.zeros((0, 2), np.float32), np.zeros((0, 3), np.float32), 1.0, 19, 23)
    out, den = run(im, np.zeros(0, np.float32), 1.0, cuda_device)
    assert (out == 0).all() and (den == 0).all()
    im = wl.Image(np.array([[5.3, 7.9]], np.float32), np.array([[0.25, 0.5, 0.75]], np.float32), 2.0, 33, 41)
    out, den = run(im, np.float32([0.7]), 2.0, cuda_device, k=3.0)
    ref = oracle.forward_pp(im.points, im.values, np.float32([0.7]), im.H, im.W, mode=oracle.TRUNCATED, k=3.0)
    inside = (ref["den"] > 0) & (ref["skipped"] < 1e-3)
    np.testing.assert_allclose(out[inside], np.broadcast_to(im.values[0], out[inside].shape), rtol=0, atol=1e-6)
    assert (out[~inside & (ref["skipped"] < 1e-3)] == 0).all()


def test_sigma_range_and_nonfinite_reported(cuda_device):
    import torch
    g = gmi()
    im = wl.tiny_random(14, 50, 12, 12, C=3, sigma=1.0)
    P, V = to_dev(im.points, cuda_device), to_dev(im.values, cuda_device)
    for bad, status in ((1.5, 1), (0.0, 1), (-0.5, 1), (np.nan, 2), (np.inf, 2)):
        sig = np.full(im.N, 0.5, np.float32)
        sig[7] = bad
        with pytest.raises(g.GmiError) as e:
            g.interpolate_pp(P, V, to_dev(sig, cuda_device), 1.0, 12, 12, check=True, mode="truncated")
        assert e.value.status == status, (bad, e.value.status)
    # the same call through the C-ABI in exact mode
    lib = g.lib()
    from paper_2012_13257_b300 import _lib
    p = _lib.make_params(1.0, 6.0, _lib.MODE_EXACT, 0, 0, 0)
    sig = to_dev(np.full(im.N, 0.5, np.float32), cuda_device)
    out = to_dev(np.zeros((12, 12, 3), np.float32), cuda_device)
    n = ctypes.c_size_t(0)
    assert lib.gmi_workspace_size(im.N, 3, 12, 12, ctypes.byref(p), ctypes.byref(n)) == 0
    ws = to_dev(np.zeros(n.value + 256, np.uint8), cuda_device)
    base = (ws.data_ptr() + 255) // 256 * 256
    st = lib.gmi_forward_pp(P.data_ptr(), V.data_ptr(), sig.data_ptr(), im.N, 3, 12, 12, ctypes.byref(p),
                            out.data_ptr(), None, base, n.value, None)
    assert st == 0
    ref = oracle.forward_pp(im.points, im.values, np.full(im.N, 0.5, np.float32), 12, 12, mode=oracle.EXACT)
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - ref["image"]).max() <= TOL_FWD


def test_graph_replay(cuda_device):
    import torch
    g = gmi()
    im = wl.tiny_random(15, 900, 64, 64, C=3, sigma=1.2, clustered=True)
    sig = wl.point_sigmas(16, im.N, 0.4, 1.2)
    P, V, S = to_dev(im.points, cuda_device), to_dev(im.values, cuda_device), to_dev(sig, cuda_device)
    out = torch.empty((64, 64, 3), device=cuda_device)
    ref = g.interpolate_pp(P, V, S, 1.2, 64, 64, radius_sigmas=4.0, mode="truncated").cpu().numpy()
    for step in range(3):
        S.mul_(0.99 if step else 1.0)   # new contents, same buffers: replay reads them
        got = g.interpolate_pp(P, V, S, 1.2, 64, 64, radius_sigmas=4.0, graph=True, out=out, mode="truncated")
        want = g.interpolate_pp(P, V, S, 1.2, 64, 64, radius_sigmas=4.0, mode="truncated")
        torch.cuda.synchronize()
        np.testing.assert_allclose(got.cpu().numpy(), want.cpu().numpy(), rtol=0, atol=2e-6)
    assert np.abs(out.cpu().numpy() - ref).max() > 0   # the sigmas did change the image


def test_full_size_sampled(cuda_device):
    """The 512^2 -> 1024^2 upsampling workload with sigma_i log-uniform in
    [0.5, 1.5] px (bound 1.5, k = 3), checked on a pixel sample."""
    im = wl.upsample_1024()
    sig = wl.point_sigmas(17, im.N, 0.5, 1.5)
    out, den = run(im, sig, 1.5, cuda_device, k=3.0)
    pix = sample_pixels(im.points, im.H, im.W, n_far=0)
    ref = oracle.forward_pp(im.points, im.values, sig, im.H, im.W, mode=oracle.TRUNCATED, k=3.0, pixels=pix)
    decided = ref["skipped"] < 1e-3
    got = out.reshape(-1, 3)[pix]
    assert np.abs(got - ref["image"])[decided].max() <= TOL_FWD
    assert np.isfinite(out).all() and out.min() >= -1e-6 and out.max() <= 1 + 1e-6


def gpu_grads(im, sig, bound, g_up, dev, k, **kw):
    import torch
    G = gmi()
    P, V, S = to_dev(im.points, dev), to_dev(im.values, dev), to_dev(sig, dev)
    img, den = G.interpolate_pp(P, V, S, bound, im.H, im.W, radius_sigmas=k, return_aux=True, **kw, mode="truncated")
    gp, gv, gs = G.interpolate_backward_pp(P, V, S, bound, im.H, im.W, img, den, to_dev(g_up, dev),
                                           radius_sigmas=k, check=True, **kw, mode="truncated")
    torch.cuda.synchronize()
    return gp.cpu().numpy(), gv.cpu().numpy(), gs.cpu().numpy()


def assert_grads(got, ref, tol=TOL_BWD):
    for name, a, b in zip(("points", "values", "sigmas"), got, (ref["points"], ref["values"], ref["sigmas"])):
        scale = np.abs(b).max()
        err = np.abs(a.astype(np.float64) - b).max()
        assert np.isfinite(a).all(), name
        assert err <= tol * max(scale, 1e-30), "%s: max err %.3g vs scale %.3g" % (name, err, scale)


@pytest.mark.parametrize("case", CASES, ids=lambda c: "s%d_N%d_%dx%d_C%d" % c[:5])
def test_backward_matches_oracle(cuda_device, case):
    seed, N, H, W, C, lo, hi, k, clustered = case
    im = wl.tiny_random(seed, N, H, W, C=C, sigma=hi, clustered=clustered, margin=2.0 if not clustered else 0.0)
    sig = wl.point_sigmas(seed + 7, N, lo, hi)
    g = np.random.default_rng(seed + 100).standard_normal((H, W, C)).astype(np.float32)
    ref = oracle.backward_pp(im.points, im.values, sig, H, W, g, mode=oracle.TRUNCATED, k=k)
    assert_grads(gpu_grads(im, sig, hi, g, cuda_device, k), ref)


@pytest.mark.parametrize("variant", [2, 3])
def test_backward_variants(cuda_device, variant):
    seed, N, H, W, C, lo, hi, k, clustered = CASES[1]
    im = wl.tiny_random(seed, N, H, W, C=C, sigma=hi, clustered=clustered)
    sig = wl.point_sigmas(seed + 7, N, lo, hi)
    g = np.random.default_rng(seed + 100).standard_normal((H, W, C)).astype(np.float32)
    ref = oracle.backward_pp(im.points, im.values, sig, H, W, g, mode=oracle.TRUNCATED, k=k)
    assert_grads(gpu_grads(im, sig, hi, g, cuda_device, k, variant=variant), ref)


def test_backward_is_deterministic(cuda_device):
    """Given the same forward outputs, the backward writes each gradient from
    one thread: bitwise the same on every run (the forward itself may differ
    in the last bits, its split tiles adding partial sums in any order)."""
    import torch
    G = gmi()
    im = wl.tiny_random(18, 900, 64, 64, C=3, sigma=1.5, clustered=True)
    sig = wl.point_sigmas(19, im.N, 0.5, 1.5)
    g = to_dev(np.random.default_rng(18).standard_normal((64, 64, 3)).astype(np.float32), cuda_device)
    P, V, S = to_dev(im.points, cuda_device), to_dev(im.values, cuda_device), to_dev(sig, cuda_device)
    img, den = G.interpolate_pp(P, V, S, 1.5, 64, 64, radius_sigmas=3.0, return_aux=True, mode="truncated")
    a = G.interpolate_backward_pp(P, V, S, 1.5, 64, 64, img, den, g, radius_sigmas=3.0, mode="truncated")
    b = G.interpolate_backward_pp(P, V, S, 1.5, 64, 64, img, den, g, radius_sigmas=3.0, mode="truncated")
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_autograd_op(cuda_device):
    import torch
    G = gmi()
    seed, N, H, W, C, lo, hi, k, clustered = CASES[0]
    im = wl.tiny_random(seed, N, H, W, C=C, sigma=hi)
    sig = wl.point_sigmas(seed + 7, N, lo, hi)
    g = np.random.default_rng(seed + 100).standard_normal((H, W, C)).astype(np.float32)
    P = to_dev(im.points, cuda_device).requires_grad_(True)
    V = to_dev(im.values, cuda_device).requires_grad_(True)
    S = to_dev(sig, cuda_device).requires_grad_(True)
    img = G.gmi_interpolate_pp(P, V, S, hi, H, W, radius_sigmas=k, mode="truncated")
    (img * to_dev(g, cuda_device)).sum().backward()
    ref = oracle.backward_pp(im.points, im.values, sig, H, W, g, mode=oracle.TRUNCATED, k=k)
    assert_grads((P.grad.cpu().numpy(), V.grad.cpu().numpy(), S.grad.cpu().numpy()), ref)


def test_sigma_descent_lowers_loss(cuda_device):
    """A few gradient steps on the per-point sigmas alone lower a
    reconstruction loss (the gradient points downhill)."""
    import torch
    G = gmi()
    im = wl.tiny_random(20, 400, 48, 48, C=3, sigma=2.0)
    P, V = to_dev(im.points, cuda_device), to_dev(im.values, cuda_device)
    target = G.interpolate_pp(P, V, to_dev(np.full(im.N, 1.0, np.float32), cuda_device), 2.0, 48, 48,
                              radius_sigmas=4.0, mode="truncated").detach()
    S = to_dev(wl.point_sigmas(21, im.N, 0.6, 1.8), cuda_device).requires_grad_(True)
    losses = []
    for _ in range(5):
        img = G.gmi_interpolate_pp(P, V, S, 2.0, 48, 48, radius_sigmas=4.0, mode="truncated")
        loss = ((img - target) ** 2).mean()
        losses.append(float(loss.detach()))
        S.grad = None
        loss.backward()
        with torch.no_grad():
            S -= 20.0 * S.grad
            S.clamp_(0.2, 2.0)
    assert losses[-1] < losses[0]


# ---------------------------------------------- axis-aligned (sx_i, sy_i) per point
def check_forward_aniso(im, sxy, bound, dev, k, **kw):
    out, den = run(im, sxy, bound, dev, k=k, **kw)
    ref = oracle.forward_aniso(im.points, im.values, sxy, im.H, im.W, mode=oracle.TRUNCATED, k=k)
    decided = ref["skipped"] < 1e-3
    assert decided.mean() > 0.99
    assert np.isfinite(out).all()
    assert np.abs(out.astype(np.float64) - ref["image"])[decided].max() <= TOL_FWD
    scaled = ref["den"] * float(bound) ** 2
    live = decided & (scaled > 0)
    assert (np.abs(den.astype(np.float64) - scaled)[live] / scaled[live]).max() <= 1e-4
    empty = (ref["den"] == 0) & decided
    assert (out[empty] == 0).all()


@pytest.mark.parametrize("case", CASES, ids=lambda c: "s%d_N%d_%dx%d_C%d" % c[:5])
@pytest.mark.parametrize("variant", [1, 2, 3])
def test_aniso_forward_matches_oracle(cuda_device, case, variant):
    seed, N, H, W, C, lo, hi, k, clustered = case
    im = wl.tiny_random(seed, N, H, W, C=C, sigma=hi, clustered=clustered, margin=2.0 if not clustered else 0.0)
    sxy = wl.point_sigmas(seed + 8, N, lo, hi, axes=2)
    check_forward_aniso(im, sxy, hi, cuda_device, k, variant=variant)


def test_aniso_equal_axes_match_isotropic(cuda_device):
    im = wl.tiny_random(31, 800, 60, 70, C=3, sigma=1.4, clustered=True)
    sig = wl.point_sigmas(32, im.N, 0.4, 1.4)
    a, da = run(im, sig, 1.4, cuda_device, k=3.0)
    b, db = run(im, np.stack([sig, sig], 1), 1.4, cuda_device, k=3.0)
    assert np.abs(a - b).max() <= 2e-6
    np.testing.assert_allclose(da, db, rtol=2e-6, atol=1e-30)


def test_aniso_range_reported(cuda_device):
    g = gmi()
    im = wl.tiny_random(33, 50, 12, 12, C=3, sigma=1.0)
    P, V = to_dev(im.points, cuda_device), to_dev(im.values, cuda_device)
    for ax, bad, status in ((0, 1.5, 1), (1, 0.0, 1), (1, np.nan, 2)):
        sxy = np.full((im.N, 2), 0.5, np.float32)
        sxy[9, ax] = bad
        with pytest.raises(g.GmiError) as e:
            g.interpolate_pp(P, V, to_dev(sxy, cuda_device), 1.0, 12, 12, check=True, mode="truncated")
        assert e.value.status == status, (ax, bad, e.value.status)
    with pytest.raises(ValueError):
        g.interpolate_pp(P, V, to_dev(np.full((im.N, 4), 0.5, np.float32), cuda_device), 1.0, 12, 12, mode="truncated")


def test_aniso_full_size_sampled(cuda_device):
    """The 1024^2 upsampling workload with sx_i, sy_i independently
    log-uniform in [0.4, 1.5] px (bound 1.5, k = 3), on a pixel sample."""
    im = wl.upsample_1024()
    sxy = wl.point_sigmas(34, im.N, 0.4, 1.5, axes=2)
    out, den = run(im, sxy, 1.5, cuda_device, k=3.0)
    pix = sample_pixels(im.points, im.H, im.W, n_far=0)
    ref = oracle.forward_aniso(im.points, im.values, sxy, im.H, im.W, mode=oracle.TRUNCATED, k=3.0, pixels=pix)
    decided = ref["skipped"] < 1e-3
    assert np.abs(out.reshape(-1, 3)[pix] - ref["image"])[decided].max() <= TOL_FWD


@pytest.mark.parametrize("case", CASES, ids=lambda c: "s%d_N%d_%dx%d_C%d" % c[:5])
def test_aniso_backward_matches_oracle(cuda_device, case):
    seed, N, H, W, C, lo, hi, k, clustered = case
    im = wl.tiny_random(seed, N, H, W, C=C, sigma=hi, clustered=clustered, margin=2.0 if not clustered else 0.0)
    sxy = wl.point_sigmas(seed + 8, N, lo, hi, axes=2)
    g = np.random.default_rng(seed + 100).standard_normal((H, W, C)).astype(np.float32)
    ref = oracle.backward_aniso(im.points, im.values, sxy, H, W, g, mode=oracle.TRUNCATED, k=k)
    ref["sigmas"] = ref["sigmas_xy"]
    got = gpu_grads(im, sxy, hi, g, cuda_device, k)
    assert got[2].shape == (N, 2)
    assert_grads(got, ref)


def test_aniso_autograd_op(cuda_device):
    import torch
    G = gmi()
    seed, N, H, W, C, lo, hi, k, clustered = CASES[2]
    im = wl.tiny_random(seed, N, H, W, C=C, sigma=hi, clustered=clustered)
    sxy = wl.point_sigmas(seed + 8, N, lo, hi, axes=2)
    g = np.random.default_rng(seed + 100).standard_normal((H, W, C)).astype(np.float32)
    P = to_dev(im.points, cuda_device).requires_grad_(True)
    V = to_dev(im.values, cuda_device).requires_grad_(True)
    S = to_dev(sxy, cuda_device).requires_grad_(True)
    img = G.gmi_interpolate_pp(P, V, S, hi, H, W, radius_sigmas=k, mode="truncated")
    (img * to_dev(g, cuda_device)).sum().backward()
    ref = oracle.backward_aniso(im.points, im.values, sxy, H, W, g, mode=oracle.TRUNCATED, k=k)
    ref["sigmas"] = ref["sigmas_xy"]
    assert_grads((P.grad.cpu().numpy(), V.grad.cpu().numpy(), S.grad.cpu().numpy()), ref)


# ---------------------------------------------- full covariance (sx_i, sy_i, rho_i) per point
def check_forward_cov(im, cov, bound, dev, k, **kw):
    out, den = run(im, cov, bound, dev, k=k, **kw)
    ref = oracle.forward_cov(im.points, im.values, cov, im.H, im.W, mode=oracle.TRUNCATED, k=k)
    decided = ref["skipped"] < 1e-3
    assert decided.mean() > 0.99
    assert np.isfinite(out).all()
    assert np.abs(out.astype(np.float64) - ref["image"])[decided].max() <= TOL_FWD
    scaled = ref["den"] * float(bound) ** 2
    live = decided & (scaled > 0)
    assert (np.abs(den.astype(np.float64) - scaled)[live] / scaled[live]).max() <= 1e-4
    empty = (ref["den"] == 0) & decided
    assert (out[empty] == 0).all()


@pytest.mark.parametrize("case", CASES, ids=lambda c: "s%d_N%d_%dx%d_C%d" % c[:5])
@pytest.mark.parametrize("variant", [1, 2, 3])
def test_cov_forward_matches_oracle(cuda_device, case, variant):
    seed, N, H, W, C, lo, hi, k, clustered = case
    im = wl.tiny_random(seed, N, H, W, C=C, sigma=hi, clustered=clustered, margin=2.0 if not clustered else 0.0)
    cov = wl.point_cov(seed + 9, N, lo, hi, rmax=0.9)
    check_forward_cov(im, cov, wl.cov_bound(cov), cuda_device, k, variant=variant)


def test_cov_zero_correlation_matches_aniso(cuda_device):
    im = wl.tiny_random(35, 800, 60, 70, C=3, sigma=1.4, clustered=True)
    cov = wl.point_cov(36, im.N, 0.4, 1.4)
    cov[:, 2] = 0.0
    a, da = run(im, cov, 1.4, cuda_device, k=3.0)
    b, db = run(im, cov[:, :2].copy(), 1.4, cuda_device, k=3.0)
    ref = oracle.forward_aniso(im.points, im.values, cov[:, :2].copy(), im.H, im.W, mode=oracle.TRUNCATED, k=3.0)
    decided = ref["skipped"] < 1e-3
    assert np.abs(a - b)[decided].max() <= 2e-6
    np.testing.assert_allclose(da[decided], db[decided], rtol=2e-6, atol=1e-30)


def test_cov_range_reported(cuda_device):
    g = gmi()
    im = wl.tiny_random(37, 50, 12, 12, C=3, sigma=1.0)
    P, V = to_dev(im.points, cuda_device), to_dev(im.values, cuda_device)
    for ax, bad, status in ((2, 0.995, 1), (2, -1.5, 1), (0, 1.2, 1), (2, np.nan, 2)):
        cov = np.tile(np.float32([0.5, 0.6, 0.3]), (im.N, 1))
        cov[11, ax] = bad
        with pytest.raises(g.GmiError) as e:
            g.interpolate_pp(P, V, to_dev(cov, cuda_device), 1.0, 12, 12, check=True, mode="truncated")
        assert e.value.status == status, (ax, bad, e.value.status)
    # sx = sy = bound with rho = 0.5: inside the box, but the ellipse's major
    # axis reaches k sqrt(1.5) bound, past the search radius
    cov = np.tile(np.float32([1.0, 1.0, 0.5]), (im.N, 1))
    with pytest.raises(g.GmiError) as e:
        g.interpolate_pp(P, V, to_dev(cov, cuda_device), 1.0, 12, 12, check=True, mode="truncated")
    assert e.value.status == 1
    g.interpolate_pp(P, V, to_dev(cov, cuda_device), wl.cov_bound(cov), 12, 12, check=True, mode="truncated")


def test_cov_full_size_sampled(cuda_device):
    """The 1024^2 upsampling workload with sx_i, sy_i log-uniform in
    [0.4, 1.5] px and rho_i uniform in [-0.9, 0.9] (bound 1.5, k = 3), on a
    pixel sample."""
    im = wl.upsample_1024()
    cov = wl.point_cov(38, im.N, 0.4, 1.5, rmax=0.9)
    out, den = run(im, cov, wl.cov_bound(cov), cuda_device, k=3.0)
    pix = sample_pixels(im.points, im.H, im.W, n_far=0)
    ref = oracle.forward_cov(im.points, im.values, cov, im.H, im.W, mode=oracle.TRUNCATED, k=3.0, pixels=pix)
    decided = ref["skipped"] < 1e-3
    assert np.abs(out.reshape(-1, 3)[pix] - ref["image"])[decided].max() <= TOL_FWD


@pytest.mark.parametrize("case", CASES, ids=lambda c: "s%d_N%d_%dx%d_C%d" % c[:5])
def test_cov_backward_matches_oracle(cuda_device, case):
    seed, N, H, W, C, lo, hi, k, clustered = case
    im = wl.tiny_random(seed, N, H, W, C=C, sigma=hi, clustered=clustered, margin=2.0 if not clustered else 0.0)
    cov = wl.point_cov(seed + 9, N, lo, hi, rmax=0.9)
    g = np.random.default_rng(seed + 100).standard_normal((H, W, C)).astype(np.float32)
    ref = oracle.backward_cov(im.points, im.values, cov, H, W, g, mode=oracle.TRUNCATED, k=k)
    ref["sigmas"] = ref["cov"]
    got = gpu_grads(im, cov, wl.cov_bound(cov), g, cuda_device, k)
    assert got[2].shape == (N, 3)
    assert_grads(got, ref)


def test_cov_backward_variants_and_determinism(cuda_device):
    import torch
    G = gmi()
    seed, N, H, W, C, lo, hi, k, clustered = CASES[1]
    im = wl.tiny_random(seed, N, H, W, C=C, sigma=hi, clustered=clustered)
    cov = wl.point_cov(seed + 9, N, lo, hi, rmax=0.9)
    g = np.random.default_rng(seed + 100).standard_normal((H, W, C)).astype(np.float32)
    ref = oracle.backward_cov(im.points, im.values, cov, H, W, g, mode=oracle.TRUNCATED, k=k)
    ref["sigmas"] = ref["cov"]
    bound = wl.cov_bound(cov)
    for variant in (2, 3):
        assert_grads(gpu_grads(im, cov, bound, g, cuda_device, k, variant=variant), ref)
    P, V, S = to_dev(im.points, cuda_device), to_dev(im.values, cuda_device), to_dev(cov, cuda_device)
    img, den = G.interpolate_pp(P, V, S, bound, H, W, radius_sigmas=k, return_aux=True, mode="truncated")
    gg = to_dev(g, cuda_device)
    a = G.interpolate_backward_pp(P, V, S, bound, H, W, img, den, gg, radius_sigmas=k, mode="truncated")
    b = G.interpolate_backward_pp(P, V, S, bound, H, W, img, den, gg, radius_sigmas=k, mode="truncated")
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_cov_autograd_op(cuda_device):
    G = gmi()
    seed, N, H, W, C, lo, hi, k, clustered = CASES[2]
    im = wl.tiny_random(seed, N, H, W, C=C, sigma=hi, clustered=clustered)
    cov = wl.point_cov(seed + 9, N, lo, hi, rmax=0.9)
    g = np.random.default_rng(seed + 100).standard_normal((H, W, C)).astype(np.float32)
    P = to_dev(im.points, cuda_device).requires_grad_(True)
    V = to_dev(im.values, cuda_device).requires_grad_(True)
    S = to_dev(cov, cuda_device).requires_grad_(True)
    img = G.gmi_interpolate_pp(P, V, S, wl.cov_bound(cov), H, W, radius_sigmas=k, mode="truncated")
    (img * to_dev(g, cuda_device)).sum().backward()
    ref = oracle.backward_cov(im.points, im.values, cov, H, W, g, mode=oracle.TRUNCATED, k=k)
    ref["sigmas"] = ref["cov"]
    assert_grads((P.grad.cpu().numpy(), V.grad.cpu().numpy(), S.grad.cpu().numpy()), ref)
