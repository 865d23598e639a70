"""The reconstruction sweep and the point-position optimisation (the paper's
sections 3.2 and 3.3 on synthetic fields): the interpolation they run matches
the oracle, and the gradient driving the optimisation matches the oracle's
analytic gradient."""
import math
import os
import sys

import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_helpers import TOL_FWD, sample_pixels, to_dev

pytestmark = pytest.mark.gpu
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def test_reconstruction_upsampling_matches_oracle(cuda_device):
    import paper_2012_13257_b300 as g
    f, side = 4, 96
    pts, vals, low, truth = wl.reconstruction_case(f, side)
    out = g.interpolate(to_dev(pts, cuda_device), to_dev(vals, cuda_device), 0.5 * f, side, side).cpu().numpy()
    pix = sample_pixels(pts, side, side)
    ref = oracle.forward(pts, vals, side, side, 0.5 * f, pixels=pix)
    assert np.abs(out.reshape(-1, 3)[pix] - ref["image"]).max() <= TOL_FWD


def test_reconstruction_sweep_runs(cuda_device):
    import bench
    r = bench.bench_reconstruction(cuda_device, side=96, factors=(2, 4))
    for key in ("x2", "x4"):
        row = r["factors"][key]
        for m in ("gmi", "nearest", "bilinear", "bicubic"):
            assert math.isfinite(row[m]) and 0.0 <= row[m] < 0.5
    # coarser sampling cannot reconstruct better
    assert r["factors"]["x4"]["gmi"] >= r["factors"]["x2"]["gmi"]


def test_point_optimisation_gradient_and_progress(cuda_device):
    import torch
    import paper_2012_13257_b300 as g
    rng = np.random.default_rng(9)
    side, n, sigma = 40, 200, 2.0
    params = wl.field_params(rng, 3)
    yy, xx = np.meshgrid(np.arange(side) + 0.5, np.arange(side) + 0.5, indexing="ij")
    target = wl.eval_field(params, np.stack([xx.ravel(), yy.ravel()], 1), float(side)).reshape(side, side, 3)
    p0 = wl.uniform_points(rng, n, side, side)
    vals = wl.eval_field(params, p0, float(side))
    T, V = to_dev(target, cuda_device), to_dev(vals, cuda_device)
    mu = to_dev(p0, cuda_device).clone().requires_grad_(True)
    out = g.gmi_interpolate(mu, V, sigma, side, side)
    loss = (out - T).abs().mean()
    loss.backward()
    # the L1 loss's upstream gradient is sign(out - target) / numel: feed the same to the oracle
    up = (torch.sign(out.detach() - T) / out.numel()).cpu().numpy()
    ref = oracle.backward(p0, vals, side, side, sigma, up)["points"]
    got = mu.grad.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-3 * np.abs(ref).max()
    # a few Adam steps lower the loss
    opt = torch.optim.Adam([mu], lr=0.05)
    first = float(loss.detach())
    for _ in range(30):
        opt.zero_grad(set_to_none=True)
        loss = (g.gmi_interpolate(mu, V, sigma, side, side) - T).abs().mean()
        loss.backward()
        opt.step()
    assert float(loss.detach()) < first
