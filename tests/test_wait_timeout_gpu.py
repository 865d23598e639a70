"""The device-side bounded waits give up cleanly.  gmi_set_wait_polls(0)
leaves every wait that may be made to give up no polls at all:

* the one-launch scan's grid barrier (single images): each block records the
  timeout and that the bin offsets are not valid, and every later kernel that
  would follow the offsets or the sorted arrays leaves at once;
* the staged near-field gather's wait on each work item's bulk copies
  (reached through a batched call, whose two-kernel scan has no barrier):
  the warp records the timeout, drains its copies still in flight and leaves.

Nothing faults or hangs: the calls return GMI_ERR_TIMEOUT under
GMI_FLAG_SYNC_CHECK, and with the default limits back the next call on the
same workspace, stream or plan is correct again (against the FP64 oracle)."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_helpers import TOL_FWD, to_dev
from paper_2012_13257_b300 import _lib

pytestmark = pytest.mark.gpu

GMI_ERR_TIMEOUT = 6


def _image():
    # a 64^2 jittered grid upsampled to 128^2 (sigma 1): every warp's window
    # (about 300 records) fits its staging buffer, so its items wait on copies
    return wl.upsample_1024(src=64)


class _Limit:
    """gmi_set_wait_polls(polls) inside the block, the defaults after it."""

    def __init__(self, polls):
        self.polls = polls

    def __enter__(self):
        assert _lib.load().gmi_set_wait_polls(self.polls) == 0

    def __exit__(self, *exc):
        assert _lib.load().gmi_set_wait_polls(-1) == 0
        return False


def _single(im, dev, gather):
    import torch
    L = _lib.load()
    p = _lib.make_params(im.sigma, flags=_lib.FLAG_SYNC_CHECK)
    p.gather = gather
    n = ctypes.c_size_t(0)
    assert L.gmi_workspace_size(im.N, im.C, im.H, im.W, ctypes.byref(p), ctypes.byref(n)) == 0
    ws = torch.empty(n.value, dtype=torch.uint8, device=dev)
    P, V = to_dev(im.points, dev), to_dev(im.values, dev)
    out = torch.empty((im.H, im.W, im.C), dtype=torch.float32, device=dev)
    den = torch.empty((im.H, im.W), dtype=torch.float32, device=dev)
    shift = torch.empty((im.H, im.W), dtype=torch.float32, device=dev)

    def forward():
        st = L.gmi_forward(P.data_ptr(), V.data_ptr(), im.N, im.C, im.H, im.W, ctypes.byref(p), out.data_ptr(),
                           den.data_ptr(), shift.data_ptr(), ws.data_ptr(), ws.numel(),
                           torch.cuda.current_stream(dev).cuda_stream)
        torch.cuda.synchronize()
        return st
    return forward, (P, V, out, den, shift, ws, p)


@pytest.mark.parametrize("gather", ["staged", "direct"])
def test_scan_barrier_gives_up_and_the_next_call_recovers(cuda_device, gather):
    im = _image()
    forward, (_, _, out, _, _, _, _) = _single(
        im, cuda_device, _lib.GATHER_STAGED if gather == "staged" else _lib.GATHER_DIRECT)
    with _Limit(0):
        assert forward() == GMI_ERR_TIMEOUT
    assert forward() == 0
    ref = oracle.forward(im.points, im.values, im.H, im.W, im.sigma)["image"]
    assert np.abs(out.cpu().numpy().astype(np.float64) - ref).max() <= TOL_FWD


def test_backward_after_a_scan_timeout_recovers(cuda_device):
    import torch
    L = _lib.load()
    im = _image()
    forward, (P, V, out, den, shift, ws, p) = _single(im, cuda_device, _lib.GATHER_STAGED)
    assert forward() == 0
    g = np.random.default_rng(9).standard_normal((im.H, im.W, im.C)).astype(np.float32)
    G = to_dev(g, cuda_device)
    gp = torch.empty((im.N, 2), dtype=torch.float32, device=cuda_device)
    gv = torch.empty((im.N, im.C), dtype=torch.float32, device=cuda_device)
    gs = torch.empty((1,), dtype=torch.float32, device=cuda_device)

    def backward():
        st = L.gmi_backward(P.data_ptr(), V.data_ptr(), im.N, im.C, im.H, im.W, ctypes.byref(p), out.data_ptr(),
                            den.data_ptr(), shift.data_ptr(), G.data_ptr(), gp.data_ptr(), gv.data_ptr(),
                            gs.data_ptr(), ws.data_ptr(), ws.numel(), torch.cuda.current_stream(cuda_device).cuda_stream)
        torch.cuda.synchronize()
        return st
    with _Limit(0):
        assert backward() == GMI_ERR_TIMEOUT
    assert backward() == 0
    ref = oracle.backward(im.points, im.values, im.H, im.W, im.sigma, g)
    for got, want in ((gp, ref["points"]), (gv, ref["values"])):
        got = got.cpu().numpy().astype(np.float64)
        assert np.abs(got - want).max() <= 1e-3 * np.abs(want).max()


def test_staged_copy_wait_gives_up_and_the_next_call_recovers(cuda_device):
    import torch
    import paper_2012_13257_b300 as gmi
    ims = [_image(), wl.upsample_1024(seed=7, src=48)]
    plan = gmi.BatchPlan(len(ims), sum(im.N for im in ims), sum(im.H * im.W for im in ims), 3, check=True)
    try:
        d = [{"points": to_dev(im.points, cuda_device), "values": to_dev(im.values, cuda_device),
              "sigma": im.sigma, "H": im.H, "W": im.W} for im in ims]
        with _Limit(0):
            with pytest.raises(_lib.GmiError) as err:
                plan.forward(d, use_graph=False)
            torch.cuda.synchronize()
        assert err.value.status == GMI_ERR_TIMEOUT
        outs = plan.forward(d, use_graph=False)
        torch.cuda.synchronize()
        for im, o in zip(ims, outs):
            ref = oracle.forward(im.points, im.values, im.H, im.W, im.sigma)["image"]
            assert np.abs(o.cpu().numpy().astype(np.float64) - ref).max() <= TOL_FWD
    finally:
        plan.close()
