"""Forward-pass parity: the CUDA path (through the C ABI, via the thin
binding) against the FP64 oracle, element by element.

Bar: max-abs error <= 1e-4 on colours in [0, 1] (exact mode); truncated mode
the same, on pixels whose result is not decided by a point lying on the
radius within rounding (the oracle reports those)."""
import math

import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_helpers import TOL_FWD, log_scaled_den, sample_pixels, to_dev

pytestmark = pytest.mark.gpu

VARIANTS = [1, 2, 3, 4]   # 4x4, 4x8, 2x4, 4x2 micro-tiles


def gmi():
    import paper_2012_13257_b300 as g
    return g


@pytest.fixture(autouse=True, params=["staged", "direct"])
def gather(request):
    """Every forward case runs through both near-field gathers (same sums)."""
    gmi().set_gather(request.param)
    yield request.param
    gmi().set_gather("auto")


def run(im, dev, **kw):
    import torch
    img, den, shift = gmi().interpolate(to_dev(im.points, dev), to_dev(im.values, dev), im.sigma, im.H, im.W,
                                        return_aux=True, check=True, **kw)
    torch.cuda.synchronize()
    return img.cpu().numpy(), den.cpu().numpy(), shift.cpu().numpy()


def assert_parity(im, out, ref, tol=TOL_FWD, mask=None):
    err = np.abs(out.astype(np.float64) - ref["image"])
    if mask is not None:
        err = err[mask]
    assert np.isfinite(out).all()
    assert err.max() <= tol, "max abs err %.3g at %s" % (err.max(), np.unravel_index(np.argmax(err), err.shape))


@pytest.mark.parametrize("variant", VARIANTS)
def test_small_uniform_full_image(cuda_device, variant):
    im = wl.small_uniform()
    out, den, shift = run(im, cuda_device, variant=variant)
    ref = oracle.forward(im.points, im.values, im.H, im.W, im.sigma)
    assert_parity(im, out, ref)
    np.testing.assert_allclose(log_scaled_den(den, shift, im.sigma),
                               log_scaled_den(ref["den"], ref["shift"], im.sigma), rtol=0, atol=1e-5)


CASES = [  # (seed, N, H, W, C, sigma, margin, clustered)
    (1, 64, 16, 16, 3, 1.0, 0.0, False),
    (2, 500, 37, 53, 3, 0.7, 3.0, False),
    (3, 200, 29, 31, 1, 2.5, 0.0, False),
    (4, 300, 40, 24, 2, 0.45, 10.0, False),
    (5, 1, 13, 7, 4, 1.3, 0.0, False),
    (6, 2, 9, 17, 3, 0.9, 0.0, False),
    (7, 50, 1, 100, 3, 1.0, 0.0, False),
    (8, 50, 100, 1, 3, 1.0, 0.0, False),
    (9, 5, 1, 1, 3, 1.0, 2.0, False),
    (10, 800, 64, 96, 3, 0.5, 0.0, True),
    (11, 800, 64, 96, 3, 2.0, 0.0, True),
    (12, 3000, 131, 67, 4, 1.1, 1.0, True),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "s%d_N%d_%dx%d_C%d" % c[:5])
@pytest.mark.parametrize("variant", VARIANTS)
def test_random_ragged_exact(cuda_device, case, variant):
    seed, N, H, W, C, s, margin, clustered = case
    im = wl.tiny_random(seed, N, H, W, C=C, sigma=s, margin=margin, clustered=clustered)
    out, den, shift = run(im, cuda_device, variant=variant)
    ref = oracle.forward(im.points, im.values, H, W, im.sigma)
    assert_parity(im, out, ref)
    np.testing.assert_allclose(log_scaled_den(den, shift, im.sigma),
                               log_scaled_den(ref["den"], ref["shift"], im.sigma), rtol=0, atol=1e-4)


@pytest.mark.parametrize("bin_px", [1, 2, 4, 16, 64])
def test_bin_sizes(cuda_device, bin_px):
    im = wl.tiny_random(21, 700, 50, 70, C=3, sigma=0.8, clustered=True)
    out, _, _ = run(im, cuda_device, bin_px=bin_px)
    assert_parity(im, out, oracle.forward(im.points, im.values, im.H, im.W, im.sigma))


@pytest.mark.parametrize("sigma", [0.5, 1.0])
def test_far_field_corner_cluster(cuda_device, sigma):
    """Points only in a corner: most pixels lie hundreds of pixels from the
    nearest point, where only a razor-thin shell of points matters and
    float32 d^2 alone cannot resolve the Voronoi-edge blends."""
    rng = np.random.default_rng(7)
    pts = rng.uniform(0, 12, (40, 2)).astype(np.float32)
    vals = rng.uniform(0, 1, (40, 3)).astype(np.float32)
    im = wl.Image(pts, vals, sigma, 200, 260)
    out, den, shift = run(im, cuda_device)
    ref = oracle.forward(im.points, im.values, im.H, im.W, im.sigma)
    assert ref["shift"].max() > 200.0 ** 2
    assert_parity(im, out, ref)


@pytest.mark.parametrize("variant", VARIANTS)
def test_truncated_mode(cuda_device, variant):
    im = wl.tiny_random(31, 400, 45, 61, C=3, sigma=0.9, clustered=True)
    k = 3.0
    out, den, _ = run(im, cuda_device, mode="truncated", radius_sigmas=k, variant=variant)
    ref = oracle.forward(im.points, im.values, im.H, im.W, im.sigma, mode=oracle.TRUNCATED, k=k)
    decided = ref["skipped"] < 1e-3   # a point on the radius would decide the result
    assert decided.mean() > 0.99
    assert_parity(im, out, ref, mask=decided)
    empty = ref["den"] == 0
    assert empty.any()
    assert (out[empty & decided] == 0).all()


def test_empty_point_set(cuda_device):
    im = wl.Image(np.zeros((0, 2), np.float32), np.zeros((0, 3), np.float32), 1.0, 19, 23)
    out, den, shift = run(im, cuda_device)
    assert (out == 0).all() and (den == 0).all()


def test_single_point_constant(cuda_device):
    im = wl.Image(np.array([[5.3, 7.9]], np.float32), np.array([[0.25, 0.5, 0.75]], np.float32), 0.6, 33, 41)
    out, _, _ = run(im, cuda_device)
    np.testing.assert_allclose(out, np.broadcast_to(im.values[0], out.shape), rtol=0, atol=1e-6)


def test_permutation_invariance(cuda_device):
    im = wl.tiny_random(41, 900, 48, 48, C=3, sigma=1.2, clustered=True)
    perm = np.random.default_rng(1).permutation(im.N)
    a, _, _ = run(im, cuda_device)
    b, _, _ = run(wl.Image(im.points[perm], im.values[perm], im.sigma, im.H, im.W), cuda_device)
    assert np.abs(a - b).max() <= 1e-6


def test_nonfinite_input_reported(cuda_device):
    g = gmi()
    im = wl.tiny_random(51, 30, 8, 8, C=3)
    pts = im.points.copy()
    pts[3, 0] = np.nan
    with pytest.raises(g.GmiError) as e:
        g.interpolate(to_dev(pts, cuda_device), to_dev(im.values, cuda_device), 1.0, 8, 8, check=True)
    assert e.value.status == 2


def test_upsample_1024_sampled(cuda_device):
    """The 512^2 -> 1024^2 upsampling workload at full size, in the launch
    configurations the benchmark times (plain launches, the cached graph
    captured then replayed, and the host-buffer call with its graph),
    checked on a pixel sample."""
    import torch
    im = wl.upsample_1024()
    out, den, shift = run(im, cuda_device)
    pix = sample_pixels(im.points, im.H, im.W)
    ref = oracle.forward(im.points, im.values, im.H, im.W, im.sigma, pixels=pix)
    got = out.reshape(-1, 3)[pix]
    err = np.abs(got - ref["image"]).max()
    assert err <= TOL_FWD, err
    # every pixel is finite and inside the colour range (convexity)
    assert np.isfinite(out).all() and out.min() >= -1e-6 and out.max() <= 1 + 1e-6
    P, V = to_dev(im.points, cuda_device), to_dev(im.values, cuda_device)
    dout = torch.empty((im.H, im.W, 3), dtype=torch.float32, device=cuda_device)
    hP, hV = torch.as_tensor(im.points).pin_memory(), torch.as_tensor(im.values).pin_memory()
    hout = torch.empty((im.H, im.W, 3), dtype=torch.float32).pin_memory()
    for _ in range(2):   # capture, then replay
        gmi().interpolate(P, V, im.sigma, im.H, im.W, out=dout, graph=True)
        gmi().interpolate_host(hP, hV, im.sigma, im.H, im.W, out=hout, graph=True)
    torch.cuda.synchronize()
    for img in (dout.cpu().numpy(), hout.numpy()):
        assert np.abs(img.reshape(-1, 3)[pix] - ref["image"]).max() <= TOL_FWD


def test_batched_images_sampled_single_launches(cuda_device):
    """Three images of the uneven clustered batch at full size, one launch
    each, checked on pixel samples that include the far field."""
    imgs = wl.batched_uneven()
    for im in imgs[:3]:
        out, _, _ = run(im, cuda_device)
        pix = sample_pixels(im.points, im.H, im.W, n_random=1024, n_border=256)
        ref = oracle.forward(im.points, im.values, im.H, im.W, im.sigma, pixels=pix)
        err = np.abs(out.reshape(-1, 3)[pix] - ref["image"]).max()
        assert err <= TOL_FWD, (im.H, im.W, im.sigma, err)


@pytest.mark.parametrize("variant", VARIANTS)
def test_dense_blob_split_tiles(cuda_device, variant):
    """A very dense blob with a wide sigma gives each thread thousands of
    candidates, so warp tiles are split into several work items whose partial
    sums are reduced at the end; the result must not change."""
    rng = np.random.default_rng(99)
    n = 12000
    pts = np.concatenate([rng.uniform(20, 36, (n, 2)), rng.uniform(0, 64, (200, 2))]).astype(np.float32)
    vals = rng.uniform(0, 1, (pts.shape[0], 3)).astype(np.float32)
    im = wl.Image(pts, vals, 1.6, 64, 72)
    out, den, shift = run(im, cuda_device, variant=variant)
    ref = oracle.forward(im.points, im.values, im.H, im.W, im.sigma)
    assert_parity(im, out, ref)
    np.testing.assert_allclose(log_scaled_den(den, shift, im.sigma),
                               log_scaled_den(ref["den"], ref["shift"], im.sigma), rtol=0, atol=1e-4)


def test_graph_replay(cuda_device):
    """GMI_FLAG_GRAPH: the first call captures the launch sequence, later
    calls on the same buffers replay it.  Replays read the buffers' current
    contents (values changed in place change the result), new buffers get a
    graph of their own, and inside an outer capture the flag is ignored.
    (Split warp tiles add their partial sums with float atomics in a varying
    order, so two runs agree to rounding, not bitwise.)"""
    import torch
    g = gmi()

    def same(a, b):
        return torch.allclose(a, b, rtol=0, atol=2e-6)

    im = wl.tiny_random(7, 3000, 70, 90, sigma=1.1)
    P, V = to_dev(im.points, cuda_device), to_dev(im.values, cuda_device)
    plain = g.interpolate(P, V, im.sigma, im.H, im.W)
    out = torch.empty_like(plain)
    for _ in range(3):
        g.interpolate(P, V, im.sigma, im.H, im.W, graph=True, out=out)
        torch.cuda.synchronize()
        assert same(out, plain)
    ref = oracle.forward(im.points, im.values, im.H, im.W, im.sigma)
    assert np.abs(out.cpu().numpy() - ref["image"]).max() <= TOL_FWD
    # in-place change of the inputs: the replay sees it
    V.mul_(0.5)
    g.interpolate(P, V, im.sigma, im.H, im.W, graph=True, out=out)
    torch.cuda.synchronize()
    ref2 = oracle.forward(im.points, (im.values * np.float32(0.5)).astype(np.float32), im.H, im.W, im.sigma)
    assert np.abs(out.cpu().numpy() - ref2["image"]).max() <= TOL_FWD
    # another output buffer: its own graph
    out2 = torch.empty_like(plain)
    g.interpolate(P, V, im.sigma, im.H, im.W, graph=True, out=out2)
    torch.cuda.synchronize()
    assert same(out2, out)
    # inside a torch graph capture the flag is ignored and the kernels are captured
    s = torch.cuda.Stream()
    out3 = torch.empty_like(plain)
    with torch.cuda.stream(s):
        g.interpolate(P, V, im.sigma, im.H, im.W, out=out3)
    torch.cuda.synchronize()
    gr = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gr, stream=s):
        g.interpolate(P, V, im.sigma, im.H, im.W, graph=True, out=out3)
    out3.zero_()
    gr.replay()
    torch.cuda.synchronize()
    assert same(out3, out)


def test_graph_replay_switches_the_far_field_on_and_off(cuda_device):
    """One replayed graph, the same buffers: points spread over the frame (no
    far-field micro-tile: the far kernel finds an empty queue) and then,
    written in place, squeezed into a corner (most micro-tiles far, and the
    summed-area table gets built), then spread again; each replay matches the
    oracle."""
    import torch
    g = gmi()
    rng = np.random.default_rng(61)
    H, W, n = 120, 150, 4000
    spread = np.stack([rng.uniform(0, W, n), rng.uniform(0, H, n)], 1).astype(np.float32)
    corner = rng.uniform(0, 10, (n, 2)).astype(np.float32)
    vals = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    P, V = to_dev(spread, cuda_device), to_dev(vals, cuda_device)
    out = torch.empty((H, W, 3), device=cuda_device)
    shift = torch.empty((H, W), device=cuda_device)
    for pts in (spread, corner, spread, corner):
        P.copy_(torch.as_tensor(pts, device=cuda_device))
        g.interpolate(P, V, 0.8, H, W, graph=True, out=out)
        torch.cuda.synchronize()
        ref = oracle.forward(pts, vals, H, W, 0.8)
        assert np.abs(out.cpu().numpy() - ref["image"]).max() <= TOL_FWD
        # far field: nearest squared distance beyond 100 / kappa, kappa = log2(e) / (2 sigma^2)
        far = ref["shift"] > 100.0 * 2 * 0.8 ** 2 / math.log2(math.e)
        assert far.any() == (pts is corner)


def test_graph_cache_evicts_and_recaptures(cuda_device):
    """More distinct (buffer, size) keys than the graph cache holds (32): the
    least recently used graphs are dropped, a dropped key is captured again
    on its next call, and every call matches the plain launches."""
    import torch
    g = gmi()
    im = wl.tiny_random(5, 600, 40, 56, sigma=0.9)
    P, V = to_dev(im.points, cuda_device), to_dev(im.values, cuda_device)
    plain = g.interpolate(P, V, im.sigma, im.H, im.W)
    outs = [torch.empty_like(plain) for _ in range(40)]
    for rnd in range(2):   # the second round finds the first keys evicted
        for o in outs:
            o.zero_()
            g.interpolate(P, V, im.sigma, im.H, im.W, graph=True, out=o)
        torch.cuda.synchronize()
        for o in outs:
            assert torch.allclose(o, plain, rtol=0, atol=2e-6)
