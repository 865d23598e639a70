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


def _submit_all(srv, reqs, device=None):
    """Submits every request (host pinned buffers, or device tensors when
    `device` is given); returns (ids, outputs)."""
    import torch
    ids, outs = [], []
    for im in reqs:
        if device is None:
            P = torch.as_tensor(im.points).pin_memory()
            V = torch.as_tensor(im.values).pin_memory()
            O = torch.empty((im.H, im.W, 3), dtype=torch.float32).pin_memory()
            ids.append(srv.submit(P, V, im.sigma, im.H, im.W, O))
        else:
            P, V = to_dev(im.points, device), to_dev(im.values, device)
            O = torch.empty((im.H, im.W, 3), dtype=torch.float32, device=device)
            ids.append(srv.submit_device(P, V, im.sigma, im.H, im.W, O))
        outs.append(O)
    return ids, outs


def test_serving_scale_mix(cuda_device, tmp_path):
    """Requests of the serving workload's sizes (sides up to 2048, up to four
    million points) mixed with small ones: each result equals the request run
    alone, one large request's pixels equal the FP64 oracle, at least two
    batches were on the GPU at once, and the per-request log orders every
    request's submit <= admit <= launch <= done."""
    import json
    import oracle
    from gpu_helpers import sample_pixels
    G = gmi()
    big = [wl.tiny_random(501, 4_000_000, 2048, 2048, C=3, sigma=1.3, clustered=False),
           wl.tiny_random(502, 900_000, 1536, 2048, C=3, sigma=0.8, clustered=True),
           wl.tiny_random(503, 1_800_000, 1800, 1024, C=3, sigma=1.9, clustered=True)]
    reqs = []
    small = requests(12, seed=7)
    for k in range(3):   # large ones between small ones, so batches of mixed sizes form
        reqs.append(big[k])
        reqs.extend(small[4 * k:4 * k + 4])
    srv = G.Server(budget_bytes=8 << 30, max_batch_images=4, max_batch_pixels=1 << 23, n_streams=2)
    log = tmp_path / "requests.jsonl"
    srv.set_log(str(log))
    ids, outs = _submit_all(srv, reqs)
    for i in ids:
        srv.wait(i, timeout_ms=120000)
    c = srv.counters()
    srv.set_log(None)
    srv.close()
    assert c["completed"] == len(reqs)
    assert c["launches"] < len(reqs)
    assert c["max_in_flight"] >= 2, c
    for im, O in zip(reqs, outs):
        assert np.abs(O.numpy() - alone(im, cuda_device)).max() <= TOL_FWD
    im = big[1]
    pix = sample_pixels(im.points, im.H, im.W, n_random=256, n_border=64, n_tiles=1, n_far=32, seed=3)
    ref = oracle.forward(im.points, im.values, im.H, im.W, im.sigma, pixels=pix)["image"]
    got = outs[next(k for k, r in enumerate(reqs) if r is im)].numpy().reshape(-1, 3)[pix]
    assert np.abs(got - ref).max() <= TOL_FWD
    lines = [json.loads(l) for l in log.read_text().splitlines()]
    assert sorted(l["id"] for l in lines) == sorted(ids)
    for l in lines:
        assert l["status"] == 0 and l["submit"] <= l["admit"] <= l["launch"] <= l["done"], l


def test_device_requests_equal_alone(cuda_device):
    """Requests whose buffers are device tensors (no copies, no pool memory),
    mixed with host requests, equal the same requests run alone."""
    G = gmi()
    dreqs = requests(10, seed=11)
    hreqs = requests(6, seed=12)
    srv = G.Server(budget_bytes=2 << 30, max_batch_images=6, max_batch_pixels=1 << 18, n_streams=2)
    dids, douts = _submit_all(srv, dreqs, device=cuda_device)
    hids, houts = _submit_all(srv, hreqs)
    for i in dids + hids:
        srv.wait(i, timeout_ms=60000)
    c = srv.counters()
    srv.close()
    assert c["completed"] == len(dreqs) + len(hreqs)
    for im, O in zip(dreqs, douts):
        assert np.abs(O.cpu().numpy() - alone(im, cuda_device)).max() <= TOL_FWD
    for im, O in zip(hreqs, houts):
        assert np.abs(O.numpy() - alone(im, cuda_device)).max() <= TOL_FWD


def test_device_request_rejects_host_buffers(cuda_device):
    import torch
    from paper_2012_13257_b300 import _lib
    import ctypes
    G = gmi()
    srv = G.Server(budget_bytes=1 << 30, max_batch_images=4, max_batch_pixels=1 << 16, n_streams=1)
    P, V = torch.zeros((10, 2)), torch.zeros((10, 3))
    O = torch.zeros((8, 8, 3))
    rid = ctypes.c_uint64(0)
    st = _lib.load().gmi_server_submit_device(srv._h, P.data_ptr(), V.data_ptr(), 10, 8, 8, 1.0, O.data_ptr(),
                                             ctypes.byref(rid))
    assert st == 1   # GMI_ERR_INVALID_ARG: not device memory
    srv.close()
