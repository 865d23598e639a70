"""The forward pass from host buffers (gmi_forward_host): the uploads, the
pipeline and the download through one C-ABI call, against the FP64 oracle
and against gmi_forward on device buffers (same kernels, same inputs), with
and without graph replay, pinned and pageable buffers."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_helpers import TOL_FWD, to_dev

pytestmark = pytest.mark.gpu


def gmi():
    import paper_2012_13257_b300 as g
    return g


def host(a, pin):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(a))
    return t.pin_memory() if pin else t


@pytest.mark.parametrize("pin", [True, False])
@pytest.mark.parametrize("graph", [False, True])
def test_host_call_matches_oracle_and_device_call(cuda_device, pin, graph):
    import torch
    im = wl.small_uniform()
    out = host(np.zeros((im.H, im.W, 3), np.float32), pin)
    for _ in range(2):   # the second call replays the graph
        gmi().interpolate_host(host(im.points, pin), host(im.values, pin), im.sigma, im.H, im.W, out=out,
                               graph=graph, check=True)
    ref = oracle.forward(im.points, im.values, im.H, im.W, im.sigma)["image"]
    assert np.abs(out.numpy().astype(np.float64) - ref).max() <= TOL_FWD
    dev = gmi().interpolate(to_dev(im.points, cuda_device), to_dev(im.values, cuda_device), im.sigma, im.H, im.W)
    torch.cuda.synchronize()
    # same kernels on the same inputs: equal up to the run-to-run order of the
    # split tiles' partial sums (last-bit differences)
    np.testing.assert_allclose(out.numpy(), dev.cpu().numpy(), rtol=0, atol=1e-6)


@pytest.mark.parametrize("C,mode", [(1, "exact"), (2, "truncated"), (4, "exact"), (3, "truncated")])
def test_host_call_channels_and_modes(cuda_device, C, mode):
    im = wl.tiny_random(12, 3000, 131, 67, C=C, sigma=1.1, margin=1.0, clustered=True)
    k = 3.0 if mode == "truncated" else 6.0
    out = gmi().interpolate_host(host(im.points, True), host(im.values, True), im.sigma, im.H, im.W,
                                 radius_sigmas=k, mode=mode, graph=True, check=True)
    ref = oracle.forward(im.points, im.values, im.H, im.W, im.sigma,
                         mode=oracle.TRUNCATED if mode == "truncated" else oracle.EXACT, k=k)
    err = np.abs(out.numpy().astype(np.float64) - ref["image"])
    # truncated mode: skip pixels decided by a point on the radius within rounding
    decided = ref["skipped"] < 1e-3 if mode == "truncated" else np.ones((im.H, im.W), bool)
    assert decided.mean() > 0.99
    assert err[decided].max() <= TOL_FWD


def test_host_call_graph_replay_sees_new_host_contents(cuda_device):
    import torch
    im = wl.tiny_random(2, 500, 37, 53, C=3, sigma=0.7, margin=3.0)
    P, V = host(im.points, True), host(im.values, True)
    out = host(np.zeros((im.H, im.W, 3), np.float32), True)
    gmi().interpolate_host(P, V, im.sigma, im.H, im.W, out=out, graph=True, check=True)
    V.copy_(torch.as_tensor(1.0 - im.values))   # same buffers, new contents: the graph re-reads them
    gmi().interpolate_host(P, V, im.sigma, im.H, im.W, out=out, graph=True, check=True)
    ref = oracle.forward(im.points, 1.0 - im.values, im.H, im.W, im.sigma)["image"]
    assert np.abs(out.numpy().astype(np.float64) - ref).max() <= TOL_FWD


def test_host_call_empty_point_set(cuda_device):
    out = gmi().interpolate_host(host(np.zeros((0, 2), np.float32), True), host(np.zeros((0, 3), np.float32), True),
                                 1.0, 9, 7, check=True)
    assert out.shape == (9, 7, 3) and not out.numpy().any()


def test_host_call_rejects_a_small_workspace(cuda_device):
    import torch
    L = gmi().lib()
    from paper_2012_13257_b300 import _lib
    im = wl.small_uniform()
    p = _lib.make_params(im.sigma)
    need = ctypes.c_size_t(0)
    assert L.gmi_forward_host_workspace_size(im.N, 3, im.H, im.W, ctypes.byref(p), ctypes.byref(need)) == 0
    ws = torch.empty(int(need.value) - 256, dtype=torch.uint8, device=cuda_device)
    P, V = host(im.points, True), host(im.values, True)
    out = host(np.zeros((im.H, im.W, 3), np.float32), True)
    st = L.gmi_forward_host(P.data_ptr(), V.data_ptr(), im.N, 3, im.H, im.W, ctypes.byref(p), out.data_ptr(),
                            ws.data_ptr(), ws.numel(), None)
    assert st == 3   # GMI_ERR_WORKSPACE
