"""Serving loop (continuous batching): requests submitted together are
admitted as memory and stream slots free up, batched, overlapped on the GPU,
and each result must equal the same request run alone (gmi_forward) within
the forward tolerance; a budget smaller than the offered load queues
requests instead of failing them; malformed or oversized requests get their
status codes."""
import numpy as np
import pytest

import workloads as wl
from gpu_helpers import TOL_FWD, to_dev

pytestmark = pytest.mark.gpu


def gmi():
    import paper_2012_13257_b300 as g
    return g


def requests(n, seed=0, lo=16, hi=200):
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n):
        H, W = int(rng.integers(lo, hi)), int(rng.integers(lo, hi))
        N = int(rng.uniform(0.1, 1.0) * H * W)
        out.append(wl.tiny_random(seed * 1000 + r, N, H, W, C=3, sigma=float(rng.uniform(0.5, 2.0)),
                                  clustered=bool(r % 2)))
    return out


def alone(im, dev):
    return gmi().interpolate(to_dev(im.points, dev), to_dev(im.values, dev), im.sigma, im.H, im.W).cpu().numpy()


def test_mix_equals_alone(cuda_device):
    import torch
    G = gmi()
    reqs = requests(40, seed=1)
    srv = G.Server(budget_bytes=4 << 30, max_batch_images=8, max_batch_pixels=1 << 17, n_streams=3)
    outs, ids = [], []
    for im in reqs:
        P = torch.as_tensor(im.points).pin_memory()
        V = torch.as_tensor(im.values).pin_memory()
        O = torch.empty((im.H, im.W, 3), dtype=torch.float32).pin_memory()
        ids.append(srv.submit(P, V, im.sigma, im.H, im.W, O))
        outs.append(O)
    lat = [srv.wait(i, timeout_ms=60000) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs)
    assert st["launches"] < len(reqs)          # requests were batched
    assert all(l > 0 for l in lat)
    for im, O in zip(reqs, outs):
        assert np.abs(O.numpy() - alone(im, cuda_device)).max() <= TOL_FWD


def test_budget_queues_instead_of_failing(cuda_device):
    import torch
    G = gmi()
    reqs = requests(12, seed=2, lo=100, hi=160)
    # plans take most of the budget; request memory fits only a few at once
    srv = G.Server(budget_bytes=int(0.6 * (1 << 30)), max_batch_images=4, max_batch_pixels=1 << 16, n_streams=2)
    outs, ids = [], []
    for im in reqs:
        O = torch.empty((im.H, im.W, 3), dtype=torch.float32)
        ids.append(srv.submit(torch.as_tensor(im.points), torch.as_tensor(im.values), im.sigma, im.H, im.W, O))
        outs.append(O)
    for i in ids:
        srv.wait(i, timeout_ms=60000)
    for im, O in zip(reqs, outs):
        assert np.abs(O.numpy() - alone(im, cuda_device)).max() <= TOL_FWD
    srv.close()


def test_status_codes(cuda_device):
    import torch
    G = gmi()
    srv = G.Server(budget_bytes=1 << 30, max_batch_images=4, max_batch_pixels=1 << 16, n_streams=1)
    O = torch.empty((300, 300, 3), dtype=torch.float32)
    with pytest.raises(G.GmiError) as e:   # larger than one batch may hold
        srv.submit(torch.zeros((10, 2)), torch.zeros((10, 3)), 1.0, 300, 300, O)
    assert e.value.status == 9
    with pytest.raises(G.GmiError) as e:
        srv.submit(torch.zeros((10, 2)), torch.zeros((10, 3)), -1.0, 8, 8, O)
    assert e.value.status == 1
    with pytest.raises(G.GmiError) as e:
        srv.wait(123456, timeout_ms=0)
    assert e.value.status == 8
    # an empty request completes with an all-zero image
    Z = torch.ones((5, 7, 3), dtype=torch.float32)
    rid = srv.submit(torch.zeros((0, 2)), torch.zeros((0, 3)), 1.0, 5, 7, Z)
    srv.wait(rid, timeout_ms=60000)
    assert float(Z.abs().max()) == 0.0
    srv.close()
