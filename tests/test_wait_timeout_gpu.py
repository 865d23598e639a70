"""The device-side bounded waits give up cleanly.  The staged near-field
gather waits on an mbarrier for each work item's bulk copies; with the wait
limit set to zero polls (gmi_set_wait_polls) every such wait gives up at once,
the warp records the timeout in the workspace's status word, drains its copies
still in flight and leaves.  Nothing faults or hangs: the call returns
GMI_ERR_TIMEOUT under GMI_FLAG_SYNC_CHECK, and with the default limit back the
next call on the same workspace and stream is correct again (against the FP64
oracle)."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_helpers import TOL_FWD, to_dev
from paper_2012_13257_b300 import _lib

pytestmark = pytest.mark.gpu

GMI_ERR_TIMEOUT = 6


def _forward(L, im, dev, ws, out):
    import torch
    p = _lib.make_params(im.sigma, flags=_lib.FLAG_SYNC_CHECK)
    p.gather = _lib.GATHER_STAGED
    P, V = to_dev(im.points, dev), to_dev(im.values, dev)
    st = L.gmi_forward(P.data_ptr(), V.data_ptr(), im.N, im.C, im.H, im.W, ctypes.byref(p), out.data_ptr(),
                       None, None, ws.data_ptr(), ws.numel(), torch.cuda.current_stream(dev).cuda_stream)
    torch.cuda.synchronize()
    return st


def test_staged_wait_gives_up_and_the_next_call_recovers(cuda_device):
    import torch
    L = _lib.load()
    # a 64^2 jittered grid upsampled to 128^2 (sigma 1): every warp's window
    # (about 300 records) fits its staging buffer, so its items wait on copies
    im = wl.upsample_1024(src=64)
    p = _lib.make_params(im.sigma)
    p.gather = _lib.GATHER_STAGED
    n = ctypes.c_size_t(0)
    assert L.gmi_workspace_size(im.N, im.C, im.H, im.W, ctypes.byref(p), ctypes.byref(n)) == 0
    ws = torch.empty(n.value, dtype=torch.uint8, device=cuda_device)
    out = torch.empty((im.H, im.W, im.C), dtype=torch.float32, device=cuda_device)
    try:
        assert L.gmi_set_wait_polls(0) == 0
        assert _forward(L, im, cuda_device, ws, out) == GMI_ERR_TIMEOUT
    finally:
        assert L.gmi_set_wait_polls(-1) == 0
    assert _forward(L, im, cuda_device, ws, out) == 0
    ref = oracle.forward(im.points, im.values, im.H, im.W, im.sigma)["image"]
    assert np.abs(out.cpu().numpy().astype(np.float64) - ref).max() <= TOL_FWD
