"""The allocation-free forward entry point, for callers that cannot allocate
device memory (a host application that owns the GPU memory pool, a loop that
must not stall on cudaMalloc/cudaFree, a binding that cannot pass a
workspace).  It is called through the C ABI and must reproduce the
workspace-based gmi_forward on two calls in a row (the second call must not
be disturbed by what the first left in the shared static scratch), in exact
and truncated mode, with and without the graph flag, and match the FP64
oracle directly (not only through gmi_forward); it must fit a problem
near its limit, refuse problems larger than its scratch, and allocate no
device memory.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_helpers import TOL_FWD, to_dev
from paper_2012_13257_b300 import _lib

pytestmark = pytest.mark.gpu

MODES = {"exact": _lib.MODE_EXACT, "truncated": _lib.MODE_TRUNCATED}


def _noalloc(im, dev, mode="exact", graph=False, bufs=None):
    import torch
    L = _lib.load()
    if bufs is None:
        bufs = (to_dev(im.points, dev), to_dev(im.values, dev),
                torch.empty((im.H, im.W, im.C), dtype=torch.float32, device=dev),
                torch.empty((im.H, im.W), dtype=torch.float32, device=dev),
                torch.empty((im.H, im.W), dtype=torch.float32, device=dev))
    P, V, out, den, shift = bufs
    flags = _lib.FLAG_SYNC_CHECK | (_lib.FLAG_GRAPH if graph else 0)
    p = _lib.make_params(im.sigma, mode=MODES[mode], flags=flags)
    st = L.gmi_forward_noalloc(P.data_ptr(), V.data_ptr(), im.N, im.C, im.H, im.W, ctypes.byref(p),
                               out.data_ptr(), den.data_ptr(), shift.data_ptr(),
                               torch.cuda.current_stream(dev).cuda_stream)
    assert st == 0, _lib.STATUS_NAMES.get(st, st)
    torch.cuda.synchronize()
    return out.cpu().numpy(), den.cpu().numpy(), shift.cpu().numpy()


def _reference(im, dev, mode="exact"):
    import torch
    import paper_2012_13257_b300 as g
    img, den, shift = g.interpolate(to_dev(im.points, dev), to_dev(im.values, dev), im.sigma, im.H, im.W,
                                    mode=mode, return_aux=True, check=True)
    torch.cuda.synchronize()
    return img.cpu().numpy(), den.cpu().numpy(), shift.cpu().numpy()


def _compare(got, ref):
    g, gden, gshift = got
    r, rden, rshift = ref
    assert np.abs(g - r).max() <= TOL_FWD
    np.testing.assert_allclose(gden, rden, rtol=1e-5, atol=0)
    np.testing.assert_allclose(gshift, rshift, rtol=1e-6, atol=0)


def _compare_oracle(got, im, mode):
    """The image against the FP64 oracle (default k = 6); in truncated mode
    only pixels that no point on the radius could decide are compared."""
    ref = oracle.forward(im.points, im.values, im.H, im.W, im.sigma,
                         mode=oracle.TRUNCATED if mode == "truncated" else oracle.EXACT, k=6.0)
    decided = ref["skipped"] < 1e-3
    assert decided.mean() > 0.99
    assert np.abs(got[0] - ref["image"])[decided].max() <= TOL_FWD


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("mode", ["exact", "truncated"])
def test_noalloc_matches_gmi_forward_on_two_calls(cuda_device, mode, graph):
    first = wl.small_uniform()
    second = wl.tiny_random(5, 3000, 97, 131, C=3, sigma=0.9, clustered=True)   # has far-field pixels
    for im in (first, second):
        got = _noalloc(im, cuda_device, mode, graph)
        _compare(got, _reference(im, cuda_device, mode))
        _compare_oracle(got, im, mode)


def test_noalloc_near_its_limit(cuda_device):
    """A 768 x 768 output from 147,456 points fits the scratch."""
    im = wl.upsample_1024(src=384)
    _compare(_noalloc(im, cuda_device), _reference(im, cuda_device))


def test_noalloc_allocates_no_device_memory(cuda_device):
    """Repeated calls leave the device's free memory where it was (the input
    and output buffers are made before the first reading)."""
    import torch
    im = wl.tiny_random(7, 2000, 120, 90, C=3, sigma=1.1, clustered=True)
    bufs = (to_dev(im.points, cuda_device), to_dev(im.values, cuda_device),
            torch.empty((im.H, im.W, im.C), dtype=torch.float32, device=cuda_device),
            torch.empty((im.H, im.W), dtype=torch.float32, device=cuda_device),
            torch.empty((im.H, im.W), dtype=torch.float32, device=cuda_device))
    _noalloc(im, cuda_device, bufs=bufs)   # first call on the device: loads the library's device code
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(cuda_device)
    for _ in range(3):
        _noalloc(im, cuda_device, bufs=bufs)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(cuda_device)
    assert free1 == free0


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
