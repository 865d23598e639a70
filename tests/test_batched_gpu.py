"""Batched forward: many uneven images in one binning pass and one persistent
gather, direct launches and replayed CUDA graphs.  Each image's result must
equal its single-image result (same kernels, same work per tile) within the
forward tolerance, and the oracle on a pixel sample."""
import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_helpers import TOL_FWD, sample_pixels, to_dev

pytestmark = pytest.mark.gpu


def gmi():
    import paper_2012_13257_b300 as g
    return g


def dev_images(imgs, dev):
    return [{"points": to_dev(im.points, dev), "values": to_dev(im.values, dev), "sigma": im.sigma,
             "H": im.H, "W": im.W} for im in imgs]


def small_batch(seed=0, B=12):
    rng = np.random.default_rng(seed)
    out = []
    for b in range(B):
        H, W = int(rng.integers(9, 90)), int(rng.integers(9, 90))
        N = int(rng.integers(0 if b == 3 else 1, 400))
        out.append(wl.tiny_random(seed * 100 + b, N, H, W, C=3, sigma=float(rng.uniform(0.5, 2.0)),
                                  clustered=bool(b % 2), margin=2.0 if b % 3 == 0 else 0.0))
    return out


@pytest.mark.parametrize("gather", ["staged", "direct"])
@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_matches_oracle_and_single(cuda_device, use_graph, gather):
    """A batch against the oracle and against single-image calls, with each
    staging choice the autotuner can pick (per plan and per call)."""
    import torch
    G = gmi()
    imgs = small_batch(1)
    plan = G.BatchPlan(32, 20000, 200000, 3, gather=gather)
    outs = plan.forward(dev_images(imgs, cuda_device), use_graph=use_graph)
    torch.cuda.synchronize()
    for im, o in zip(imgs, outs):
        got = o.cpu().numpy()
        ref = oracle.forward(im.points, im.values, im.H, im.W, im.sigma)["image"]
        assert np.abs(got - ref).max() <= TOL_FWD, (im.H, im.W, im.N)
        single = G.interpolate(to_dev(im.points, cuda_device), to_dev(im.values, cuda_device), im.sigma,
                               im.H, im.W, gather=gather).cpu().numpy()
        assert np.abs(got - single).max() <= 1e-6
    plan.close()


def test_graph_replay_with_different_batches(cuda_device):
    """One plan, graph replays with batches of different counts and shapes."""
    import torch
    G = gmi()
    plan = G.BatchPlan(32, 20000, 200000, 3)
    for seed, B in ((2, 10), (3, 5), (4, 16), (5, 1), (6, 12)):
        imgs = small_batch(seed, B)
        outs = plan.forward(dev_images(imgs, cuda_device), use_graph=True)
        torch.cuda.synchronize()
        for im, o in zip(imgs, outs):
            ref = oracle.forward(im.points, im.values, im.H, im.W, im.sigma)["image"]
            assert np.abs(o.cpu().numpy() - ref).max() <= TOL_FWD, (seed, im.H, im.W)
    plan.close()


def test_capacity_errors(cuda_device):
    G = gmi()
    plan = G.BatchPlan(2, 1000, 5000, 3)
    imgs = small_batch(7, 3)
    with pytest.raises(G.GmiError) as e:
        plan.forward(dev_images(imgs, cuda_device))
    assert e.value.status == 9
    big = [wl.tiny_random(8, 2000, 40, 40)]
    with pytest.raises(G.GmiError) as e:
        plan.forward(dev_images(big, cuda_device))
    assert e.value.status == 9
    plan.close()


def test_uneven_clustered_batch_sampled(cuda_device):
    """The 64-image uneven clustered workload at full size in one batched
    graph launch; every image checked on a pixel sample (incl. far field)."""
    import torch
    G = gmi()
    imgs = wl.batched_uneven()
    plan = G.BatchPlan(64, sum(i.N for i in imgs), sum(i.H * i.W for i in imgs), 3)
    outs = plan.forward(dev_images(imgs, cuda_device), use_graph=True)
    outs = plan.forward(dev_images(imgs, cuda_device), use_graph=True)   # replay
    torch.cuda.synchronize()
    for b, (im, o) in enumerate(zip(imgs, outs)):
        if b % 4:
            continue
        pix = sample_pixels(im.points, im.H, im.W, n_random=256, n_border=64, n_tiles=1, n_far=64, seed=b)
        ref = oracle.forward(im.points, im.values, im.H, im.W, im.sigma, pixels=pix)["image"]
        err = np.abs(o.cpu().numpy().reshape(-1, 3)[pix] - ref).max()
        assert err <= TOL_FWD, (b, im.H, im.W, err)
    plan.close()


def test_autotuner_picks_the_fastest_measured_candidate(cuda_device, tmp_path):
    """gmi_autotune times every (variant, bin edge), once per staging choice
    (points per stage: the staged window or none); the Python Autotuner
    records the fastest for the problem's bucket, and a forward with the
    tuned choices matches the oracle."""
    import torch
    import paper_2012_13257_b300 as G
    from paper_2012_13257_b300.autotune import Autotuner, DEFAULT_GATHERS, DEFAULT_VARIANTS, bucket
    im = wl.tiny_random(5, 6000, 120, 150, sigma=1.2)
    t = Autotuner(path=str(tmp_path / "tune.json"))
    P, V = to_dev(im.points, cuda_device), to_dev(im.values, cuda_device)
    best, times = t.tune(P, V, im.sigma, im.H, im.W, bins=(0, 2, 4), reps=3)
    assert len(times) == 3 * len(DEFAULT_VARIANTS) * len(DEFAULT_GATHERS) and all(v > 0 for v in times.values())
    assert {k.split("/")[2] for k in times} == set(DEFAULT_GATHERS)
    assert best["variant"] in DEFAULT_VARIANTS and best["bin_px"] in (0, 2, 4) and best["gather"] in DEFAULT_GATHERS
    assert best["ms"] == min(times.values())
    assert t.lookup(im.sigma, im.N / float(im.H * im.W), 3) == best
    assert bucket(im.sigma, im.N / float(im.H * im.W), 3) in t.table[t.gpu_name()]
    out = G.interpolate(P, V, im.sigma, im.H, im.W, variant=best["variant"], bin_px=best["bin_px"],
                        gather=best["gather"], check=True)
    torch.cuda.synchronize()
    ref = oracle.forward(im.points, im.values, im.H, im.W, im.sigma)["image"]
    assert np.abs(out.cpu().numpy().astype(np.float64) - ref).max() <= TOL_FWD


@pytest.mark.parametrize("C,mode,variant", [(1, "exact", 1), (2, "exact", 3), (4, "exact", 2),
                                            (3, "truncated", 1), (4, "truncated", 3)])
def test_batch_channels_modes_variants(cuda_device, C, mode, variant):
    """Batched forward (graph replay) for other channel counts, the truncated
    reading and the other micro-tiles, image by image against the oracle."""
    import torch
    G = gmi()
    rng = np.random.default_rng(40 + C + variant)
    imgs = []
    for b in range(6):
        H, W = int(rng.integers(9, 70)), int(rng.integers(9, 70))
        imgs.append(wl.tiny_random(4000 + 10 * C + variant + b, int(rng.integers(1, 300)), H, W, C=C,
                                   sigma=float(rng.uniform(0.5, 1.8)), clustered=bool(b % 2)))
    plan = G.BatchPlan(8, 3000, 40000, C, mode=mode, variant=variant)
    outs = plan.forward(dev_images(imgs, cuda_device), use_graph=True)
    torch.cuda.synchronize()
    om = oracle.TRUNCATED if mode == "truncated" else oracle.EXACT
    for im, o in zip(imgs, outs):
        ref = oracle.forward(im.points, im.values, im.H, im.W, im.sigma, mode=om)
        err = np.abs(o.cpu().numpy().astype(np.float64) - ref["image"])
        if mode == "truncated":
            err = err[ref["skipped"] < 1e-3]   # pixels not decided by a point on the radius
        assert err.max() <= TOL_FWD, (C, mode, variant, im.H, im.W, im.N)
    plan.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_degenerate_images_with_far_field(cuda_device, use_graph):
    """A batch of degenerate shapes beside far-field images (which make the
    near kernel build the summed-area table of every image): 1x1 and 1xN /
    Nx1 strips, an image without points, a point outside its frame, a
    corner cluster in a wide frame; each result equals the oracle."""
    import torch
    G = gmi()
    rng = np.random.default_rng(71)

    def img(pts, H, W, sigma=0.7):
        pts = np.asarray(pts, np.float32).reshape(-1, 2)
        vals = rng.uniform(0, 1, (pts.shape[0], 3)).astype(np.float32)
        return wl.Image(pts, vals, sigma, H, W)

    imgs = [img([[0.3, 0.6]], 1, 1),
            img(np.stack([rng.uniform(0, 97, 20), rng.uniform(0, 1, 20)], 1), 1, 97),
            img(np.stack([rng.uniform(0, 1, 15), rng.uniform(0, 83, 15)], 1), 83, 1),
            img(np.zeros((0, 2)), 17, 23),
            img([[-3.5, 4.0], [40.0, 60.0]], 31, 29, sigma=1.3),
            img(rng.uniform(0, 6, (50, 2)), 90, 140),
            img(rng.uniform(0, 6, (50, 2)) + np.float32([200, 0]), 40, 210, sigma=1.8)]
    plan = G.BatchPlan(16, 1000, 50000, 3)
    outs = plan.forward(dev_images(imgs, cuda_device), use_graph=use_graph)
    torch.cuda.synchronize()
    for im, o in zip(imgs, outs):
        ref = oracle.forward(im.points, im.values, im.H, im.W, im.sigma)["image"]
        assert np.abs(o.cpu().numpy() - ref).max() <= TOL_FWD, (im.H, im.W, im.N)
    plan.close()
