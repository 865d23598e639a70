"""The allocation-free forward entry point, for callers that cannot allocate
device memory (a host application that owns the GPU memory pool, a loop that
must not stall on cudaMalloc/cudaFree, a binding that cannot pass a
workspace).  It is called through the C ABI and must reproduce the
workspace-based gmi_forward on two calls in a row (the second call must not
be disturbed by what the first left in the shared static scratch), and must
refuse problems larger than its scratch.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import workloads as wl
from gpu_helpers import TOL_FWD, to_dev
from paper_2012_13257_b300 import _lib

pytestmark = pytest.mark.gpu


def _noalloc(im, dev):
    import torch
    L = _lib.load()
    P, V = to_dev(im.points, dev), to_dev(im.values, dev)
    out = torch.empty((im.H, im.W, im.C), dtype=torch.float32, device=dev)
    den = torch.empty((im.H, im.W), dtype=torch.float32, device=dev)
    shift = torch.empty((im.H, im.W), dtype=torch.float32, device=dev)
    p = _lib.make_params(im.sigma, flags=_lib.FLAG_SYNC_CHECK)
    st = L.gmi_forward_noalloc(P.data_ptr(), V.data_ptr(), im.N, im.C, im.H, im.W, ctypes.byref(p),
                               out.data_ptr(), den.data_ptr(), shift.data_ptr(),
                               torch.cuda.current_stream(dev).cuda_stream)
    assert st == 0, _lib.STATUS_NAMES.get(st, st)
    torch.cuda.synchronize()
    return out.cpu().numpy(), den.cpu().numpy(), shift.cpu().numpy()


def _reference(im, dev):
    import torch
    import paper_2012_13257_b300 as g
    img, den, shift = g.interpolate(to_dev(im.points, dev), to_dev(im.values, dev), im.sigma, im.H, im.W,
                                    return_aux=True, check=True)
    torch.cuda.synchronize()
    return img.cpu().numpy(), den.cpu().numpy(), shift.cpu().numpy()


def test_noalloc_matches_gmi_forward_on_two_calls(cuda_device):
    first = wl.small_uniform()
    second = wl.tiny_random(5, 3000, 97, 131, C=3, sigma=0.9, clustered=True)   # has far-field pixels
    for im in (first, second):
        got, gden, gshift = _noalloc(im, cuda_device)
        ref, rden, rshift = _reference(im, cuda_device)
        assert np.abs(got - ref).max() <= TOL_FWD
        np.testing.assert_allclose(gden, rden, rtol=1e-5, atol=0)
        np.testing.assert_allclose(gshift, rshift, rtol=1e-6, atol=0)


def test_noalloc_rejects_problems_beyond_its_scratch(cuda_device):
    L = _lib.load()
    p = _lib.make_params(1.0)
    N, H, W = 4_000_000, 2048, 2048
    n = ctypes.c_size_t(0)
    assert L.gmi_workspace_size(N, 3, H, W, ctypes.byref(p), ctypes.byref(n)) == 0
    assert n.value > _lib.NOALLOC_SCRATCH_BYTES
    # rejected before any pointer is touched
    st = L.gmi_forward_noalloc(256, 256, N, 3, H, W, ctypes.byref(p), 256, None, None, None)
    assert st == 9   # GMI_ERR_CAPACITY
