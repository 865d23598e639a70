"""Backward-pass parity: gradients w.r.t. point positions, colours and sigma
from the CUDA path against the FP64 oracle's analytic gradient (itself pinned
by finite differences and torch autograd in test_oracle.py).

Bar, per tensor: max|g_gpu - g_ref| <= 1e-3 * max|g_ref|; sigma: relative
1e-3.  Elementwise relative error is meaningless for near-zero gradients."""
import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_helpers import to_dev

pytestmark = pytest.mark.gpu

TOL_BWD = 1e-3
# entries at least this share of their tensor's largest are also checked one by one
REL_FLOOR = 1e-2


def gmi():
    import paper_2012_13257_b300 as g
    return g


def gpu_grads(im, g_up, dev, **kw):
    import torch
    G = gmi()
    P, V = to_dev(im.points, dev), to_dev(im.values, dev)
    img, den, shift = G.interpolate(P, V, im.sigma, im.H, im.W, return_aux=True, **kw)
    gp, gv, gs = G.interpolate_backward(P, V, im.sigma, im.H, im.W, img, den, shift, to_dev(g_up, dev),
                                        check=True, **kw)
    torch.cuda.synchronize()
    return gp.cpu().numpy(), gv.cpu().numpy(), float(gs.cpu().numpy()[0])


def assert_grads(got, ref, tol=TOL_BWD):
    """Per tensor: max |g - g_ref| <= tol max |g_ref|, and element by element
    |g - g_ref| <= tol |g_ref| wherever |g_ref| >= REL_FLOOR max |g_ref|
    (smaller entries carry cancellation that the first bar covers)."""
    gp, gv, gs = got
    for name, a, b in (("points", gp, ref["points"]), ("values", gv, ref["values"])):
        scale = np.abs(b).max()
        diff = np.abs(a.astype(np.float64) - b)
        err = diff.max()
        assert np.isfinite(a).all(), name
        assert err <= tol * max(scale, 1e-30), "%s: max err %.3g vs scale %.3g" % (name, err, scale)
        big = np.abs(b) >= REL_FLOOR * scale
        rel = (diff[big] / np.abs(b[big])).max() if big.any() else 0.0
        assert rel <= tol, "%s: element-wise relative err %.3g above the %.0e floor" % (name, rel, REL_FLOOR)
    assert abs(gs - ref["sigma"]) <= tol * max(abs(ref["sigma"]), 1e-6), (gs, ref["sigma"])


def test_fd_subcase(cuda_device):
    im, g = wl.fd_subcase()
    assert_grads(gpu_grads(im, g, cuda_device), oracle.backward(im.points, im.values, im.H, im.W, im.sigma, g))


CASES = [  # (seed, N, H, W, C, sigma, margin, clustered)
    (1, 64, 16, 16, 3, 1.0, 0.0, False),
    (2, 400, 37, 53, 3, 0.7, 3.0, False),
    (3, 200, 29, 31, 1, 2.5, 0.0, False),
    (4, 300, 40, 24, 2, 0.6, 8.0, False),
    (5, 600, 48, 64, 4, 1.3, 0.0, True),
    (6, 800, 64, 96, 3, 0.5, 0.0, True),
    (7, 800, 64, 96, 3, 2.0, 0.0, True),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "s%d_N%d_%dx%d_C%d" % c[:5])
def test_random_cases_exact(cuda_device, case):
    seed, N, H, W, C, s, margin, clustered = case
    im = wl.tiny_random(seed, N, H, W, C=C, sigma=s, margin=margin, clustered=clustered)
    g = np.random.default_rng(seed + 100).standard_normal((H, W, C)).astype(np.float32)
    assert_grads(gpu_grads(im, g, cuda_device), oracle.backward(im.points, im.values, H, W, im.sigma, g))


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_variants(cuda_device, variant):
    im = wl.tiny_random(9, 500, 40, 44, C=3, sigma=0.9, clustered=True)
    g = np.random.default_rng(9).standard_normal((40, 44, 3)).astype(np.float32)
    assert_grads(gpu_grads(im, g, cuda_device, variant=variant),
                 oracle.backward(im.points, im.values, im.H, im.W, im.sigma, g))


def test_far_field_corner_cluster(cuda_device):
    """Pixels hundreds of pixels from every point: the fallback kernel with
    shifted, compensated weights carries their gradient."""
    rng = np.random.default_rng(17)
    pts = rng.uniform(0, 10, (30, 2)).astype(np.float32)
    vals = rng.uniform(0, 1, (30, 3)).astype(np.float32)
    im = wl.Image(pts, vals, 0.8, 90, 120)
    g = rng.standard_normal((90, 120, 3)).astype(np.float32)
    assert_grads(gpu_grads(im, g, cuda_device), oracle.backward(im.points, im.values, im.H, im.W, im.sigma, g))


def test_truncated_mode(cuda_device):
    im = wl.tiny_random(21, 400, 45, 61, C=3, sigma=0.9, clustered=True)
    g = np.random.default_rng(21).standard_normal((45, 61, 3)).astype(np.float32)
    k = 3.0
    ref = oracle.backward(im.points, im.values, im.H, im.W, im.sigma, g, mode=oracle.TRUNCATED, k=k)
    assert_grads(gpu_grads(im, g, cuda_device, mode="truncated", radius_sigmas=k), ref)


def test_dense_blob(cuda_device):
    rng = np.random.default_rng(31)
    pts = np.concatenate([rng.uniform(10, 22, (3000, 2)), rng.uniform(0, 40, (100, 2))]).astype(np.float32)
    vals = rng.uniform(0, 1, (pts.shape[0], 3)).astype(np.float32)
    im = wl.Image(pts, vals, 1.4, 40, 40)
    g = rng.standard_normal((40, 40, 3)).astype(np.float32)
    assert_grads(gpu_grads(im, g, cuda_device), oracle.backward(im.points, im.values, im.H, im.W, im.sigma, g))


def test_autograd_function(cuda_device):
    import torch
    G = gmi()
    im, g = wl.fd_subcase(side=24, n=150)
    P = to_dev(im.points, cuda_device).requires_grad_(True)
    V = to_dev(im.values, cuda_device).requires_grad_(True)
    S = torch.tensor(im.sigma, dtype=torch.float32, device=cuda_device, requires_grad=True)
    img = G.gmi_interpolate(P, V, S, im.H, im.W)
    (img * to_dev(g, cuda_device)).sum().backward()
    ref = oracle.backward(im.points, im.values, im.H, im.W, im.sigma, g)
    assert_grads((P.grad.cpu().numpy(), V.grad.cpu().numpy(), float(S.grad)), ref)


def test_fwd_bwd_512_windows(cuda_device):
    """The 16 x 512^2 fwd+bwd workload at full size (one image here): the
    upstream gradient is kept on three 32x32 windows so the O(N*H*W) oracle
    finishes; all point gradients are compared.  With the full N(0,1)
    gradient, the colour gradients must sum to the upstream sum per channel
    (the weights of every pixel sum to one)."""
    imgs, gfull = wl.fwd_bwd_512(B=1)
    im = imgs[0]
    rng = np.random.default_rng(3)
    g = np.zeros_like(gfull[0])
    for _ in range(3):
        y, x = rng.integers(0, 512 - 32, 2)
        g[y:y + 32, x:x + 32] = gfull[0][y:y + 32, x:x + 32]
    assert_grads(gpu_grads(im, g, cuda_device), oracle.backward(im.points, im.values, im.H, im.W, im.sigma, g))
    _, gv, _ = gpu_grads(im, gfull[0], cuda_device)
    np.testing.assert_allclose(gv.astype(np.float64).sum(0), gfull[0].astype(np.float64).reshape(-1, 3).sum(0),
                               rtol=1e-4, atol=1e-2)


def test_batched_backward_matches_oracle(cuda_device):
    """Uneven images through one batched forward and one batched backward:
    every image's gradients against the oracle."""
    import torch
    G = gmi()
    rng = np.random.default_rng(77)
    imgs, ups = [], []
    for b in range(7):
        H, W = int(rng.integers(12, 40)), int(rng.integers(12, 40))
        im = wl.tiny_random(700 + b, int(rng.integers(20, 300)), H, W, C=3, sigma=float(rng.uniform(0.6, 1.8)),
                            clustered=bool(b % 2))
        imgs.append(im)
        ups.append(rng.standard_normal((H, W, 3)).astype(np.float32))
    plan = G.BatchPlan(16, 5000, 20000, 3)
    P = [to_dev(im.points, cuda_device).requires_grad_(True) for im in imgs]
    V = [to_dev(im.values, cuda_device).requires_grad_(True) for im in imgs]
    S = [torch.tensor(im.sigma, dtype=torch.float32, device=cuda_device, requires_grad=True) for im in imgs]
    outs = G.gmi_interpolate_batch(plan, P, V, S, [(im.H, im.W) for im in imgs])
    loss = sum((o * to_dev(u, cuda_device)).sum() for o, u in zip(outs, ups))
    loss.backward()
    torch.cuda.synchronize()
    for b, im in enumerate(imgs):
        ref = oracle.backward(im.points, im.values, im.H, im.W, im.sigma, ups[b])
        assert_grads((P[b].grad.cpu().numpy(), V[b].grad.cpu().numpy(), float(S[b].grad)), ref)
        fwd = oracle.forward(im.points, im.values, im.H, im.W, im.sigma)["image"]
        assert np.abs(outs[b].detach().cpu().numpy() - fwd).max() <= 1e-4
    plan.close()


def test_stacked_autograd_matches_oracle(cuda_device):
    """Equal-shaped images as stacked tensors through the stacked batched op."""
    import torch
    G = gmi()
    B, N, H, W = 5, 180, 28, 36
    ims = [wl.tiny_random(900 + b, N, H, W, C=3, sigma=0.7 + 0.2 * b, clustered=bool(b % 2)) for b in range(B)]
    rng = np.random.default_rng(5)
    ups = rng.standard_normal((B, H, W, 3)).astype(np.float32)
    P = to_dev(np.stack([im.points for im in ims]), cuda_device).requires_grad_(True)
    V = to_dev(np.stack([im.values for im in ims]), cuda_device).requires_grad_(True)
    S = torch.tensor([im.sigma for im in ims], dtype=torch.float32, device=cuda_device, requires_grad=True)
    plan = G.BatchPlan(B, B * N, B * H * W, 3)
    out = G.gmi_interpolate_stacked(plan, P, V, S, H, W)
    (out * to_dev(ups, cuda_device)).sum().backward()
    torch.cuda.synchronize()
    for b, im in enumerate(ims):
        ref = oracle.backward(im.points, im.values, H, W, im.sigma, ups[b])
        assert_grads((P.grad[b].cpu().numpy(), V.grad[b].cpu().numpy(), float(S.grad[b])), ref)
        fwd = oracle.forward(im.points, im.values, H, W, im.sigma)["image"]
        assert np.abs(out[b].detach().cpu().numpy() - fwd).max() <= 1e-4
    plan.close()


@pytest.mark.parametrize("op", ["single", "list", "stacked"])
def test_autograd_ops_free_their_buffers_each_step(cuda_device, op):
    """The autograd ops keep their tensors through save_for_backward, so a
    forward + backward step leaves no reference cycle: the device memory in
    use returns to the same level after every step without Python's cycle
    collector (a cycle through the output kept whole images alive and forced
    a device allocation per step)."""
    import gc
    import torch
    g = gmi()
    imgs = [wl.tiny_random(40 + k, 600, 48, 56, sigma=1.0) for k in range(3)]
    P = [to_dev(im.points, cuda_device).requires_grad_(True) for im in imgs]
    V = [to_dev(im.values, cuda_device).requires_grad_(True) for im in imgs]
    S = [torch.tensor(1.0, device=cuda_device, requires_grad=True) for _ in imgs]
    plan = g.BatchPlan(3, sum(im.N for im in imgs), sum(im.H * im.W for im in imgs), 3)

    def step():
        if op == "single":
            out = g.gmi_interpolate(P[0], V[0], S[0], 48, 56)
            out.sum().backward()
        elif op == "list":
            outs = g.gmi_interpolate_batch(plan, P, V, S, [(48, 56)] * 3)
            sum(o.sum() for o in outs).backward()
        else:
            out = g.gmi_interpolate_stacked(plan, torch.stack(P), torch.stack(V), torch.stack(S), 48, 56)
            out.sum().backward()

    gc.disable()
    try:
        for _ in range(3):
            step()
        torch.cuda.synchronize()
        base = torch.cuda.memory_allocated()
        for _ in range(4):
            step()
            torch.cuda.synchronize()
            assert torch.cuda.memory_allocated() == base
    finally:
        gc.enable()
        plan.close()


def test_sigma_tensors_are_read_per_tensor(cuda_device):
    """Fresh sigma tensors with new values (which the caching allocator tends
    to place at a just-freed address) are each read for what they hold; an
    in-place update of one tensor is seen too."""
    import torch
    g = gmi()
    im = wl.tiny_random(77, 500, 40, 44, sigma=1.0)
    P, V = to_dev(im.points, cuda_device), to_dev(im.values, cuda_device)
    for v in (0.8, 1.3, 0.8, 1.7, 1.1):
        S = torch.tensor(v, dtype=torch.float32, device=cuda_device)
        got = g.gmi_interpolate(P, V, S, 40, 44)
        ref = g.interpolate(P, V, float(np.float32(v)), 40, 44)
        assert torch.allclose(got, ref, rtol=0, atol=2e-6), v
        del S, got
    S = torch.tensor(0.9, dtype=torch.float32, device=cuda_device)
    g.gmi_interpolate(P, V, S, 40, 44)
    S.fill_(1.6)
    assert torch.allclose(g.gmi_interpolate(P, V, S, 40, 44), g.interpolate(P, V, float(np.float32(1.6)), 40, 44),
                          rtol=0, atol=2e-6)


@pytest.mark.parametrize("C", [1, 4])
def test_batched_backward_other_channel_counts(cuda_device, C):
    """The batched backward for one and four channels (the four-channel
    planes take two float4 per pixel) against the oracle."""
    import torch
    G = gmi()
    rng = np.random.default_rng(300 + C)
    imgs, ups = [], []
    for b in range(4):
        H, W = int(rng.integers(12, 36)), int(rng.integers(12, 36))
        imgs.append(wl.tiny_random(800 + 10 * C + b, int(rng.integers(20, 250)), H, W, C=C,
                                   sigma=float(rng.uniform(0.6, 1.6)), clustered=bool(b % 2)))
        ups.append(rng.standard_normal((H, W, C)).astype(np.float32))
    plan = G.BatchPlan(8, 2000, 8000, C)
    P = [to_dev(im.points, cuda_device).requires_grad_(True) for im in imgs]
    V = [to_dev(im.values, cuda_device).requires_grad_(True) for im in imgs]
    S = [torch.tensor(im.sigma, dtype=torch.float32, device=cuda_device, requires_grad=True) for im in imgs]
    outs = G.gmi_interpolate_batch(plan, P, V, S, [(im.H, im.W) for im in imgs])
    sum((o * to_dev(u, cuda_device)).sum() for o, u in zip(outs, ups)).backward()
    torch.cuda.synchronize()
    for b, im in enumerate(imgs):
        ref = oracle.backward(im.points, im.values, im.H, im.W, im.sigma, ups[b])
        assert_grads((P[b].grad.cpu().numpy(), V[b].grad.cpu().numpy(), float(S[b].grad)), ref)
    plan.close()
