"""gmi: Gaussian-mixture interpolation of scattered points onto a raster,
B300-native (sm_103a CUDA kernels behind the C ABI of ``libgmi.so``).

Each known point (x, y) with colour c is an isotropic 2D normal N((x, y),
sigma^2 I); every output pixel takes the normalised, density-weighted mean of
the known colours (arXiv 2012.13257, section 2, Eq. 1 and Eq. 2).

PyTorch supplies device memory and streams only; every step of the
computation runs in libgmi's kernels.  Conventions: float32 tensors on one
CUDA device, ``points[N,2]`` = (x along W, y along H) in output-pixel units,
``values[N,C]`` (C = 1..4), output ``[H,W,C]``; pixel (i, j) is evaluated at
(j + 0.5, i + 0.5).
"""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import GmiError, MODE_EXACT, MODE_TRUNCATED

__all__ = ["interpolate", "workspace_size", "GmiError", "MODE_EXACT", "MODE_TRUNCATED", "version", "lib"]


def lib():
    return _lib.load()


def version() -> str:
    return _lib.load().gmi_version().decode()


def _mode(mode) -> int:
    if mode in ("exact", MODE_EXACT, None):
        return MODE_EXACT
    if mode in ("truncated", MODE_TRUNCATED):
        return MODE_TRUNCATED
    raise ValueError("mode must be 'exact' or 'truncated'")


def workspace_size(N: int, C: int, H: int, W: int, sigma: float = 1.0, radius_sigmas: float = 6.0,
                   mode="exact", bin_px: int = 0, variant: int = 0) -> int:
    p = _lib.make_params(sigma, radius_sigmas, _mode(mode), 0, bin_px, variant)
    n = ctypes.c_size_t(0)
    _lib.check(_lib.load().gmi_workspace_size(int(N), int(C), int(H), int(W), ctypes.byref(p), ctypes.byref(n)),
               "gmi_workspace_size")
    return int(n.value)


def _check_inputs(points, values):
    import torch
    if not (isinstance(points, torch.Tensor) and isinstance(values, torch.Tensor)):
        raise TypeError("points and values must be torch tensors")
    if points.device.type != "cuda" or values.device != points.device:
        raise ValueError("points and values must live on the same CUDA device")
    if points.dtype != torch.float32 or values.dtype != torch.float32:
        raise TypeError("points and values must be float32")
    if points.dim() != 2 or points.shape[1] != 2:
        raise ValueError("points must have shape [N, 2]")
    if values.dim() != 2 or values.shape[0] != points.shape[0]:
        raise ValueError("values must have shape [N, C]")
    return points.contiguous(), values.contiguous()


def interpolate(points, values, sigma: float, H: int, W: int, *, radius_sigmas: float = 6.0,
                mode="exact", bin_px: int = 0, variant: int = 0, return_aux: bool = False,
                check: bool = False, out=None):
    """Forward pass of Eq. 1 / Eq. 2 onto an H x W raster.

    Returns the image ``[H, W, C]``; with ``return_aux`` also the per-pixel
    ``den`` and ``shift`` planes (den = sum_i exp(-(d_i^2 - shift)/(2 sigma^2))).
    ``check=True`` synchronises and raises on device-detected errors
    (non-finite inputs).  Runs on the current CUDA stream.
    """
    import torch
    points, values = _check_inputs(points, values)
    N, C = int(points.shape[0]), int(values.shape[1])
    dev = points.device
    flags = _lib.FLAG_SYNC_CHECK if check else 0
    p = _lib.make_params(sigma, radius_sigmas, _mode(mode), flags, bin_px, variant)
    L = _lib.load()
    nbytes = ctypes.c_size_t(0)
    _lib.check(L.gmi_workspace_size(N, C, int(H), int(W), ctypes.byref(p), ctypes.byref(nbytes)),
               "gmi_workspace_size")
    if out is None:
        out = torch.empty((H, W, C), dtype=torch.float32, device=dev)
    den = torch.empty((H, W), dtype=torch.float32, device=dev) if return_aux else None
    shift = torch.empty((H, W), dtype=torch.float32, device=dev) if return_aux else None
    ws = torch.empty(int(nbytes.value), dtype=torch.uint8, device=dev)
    with torch.cuda.device(dev):
        stream = torch.cuda.current_stream(dev).cuda_stream
        st = L.gmi_forward(points.data_ptr(), values.data_ptr(), N, C, int(H), int(W), ctypes.byref(p),
                           out.data_ptr(), den.data_ptr() if den is not None else None,
                           shift.data_ptr() if shift is not None else None, ws.data_ptr(),
                           int(nbytes.value), stream)
    _lib.check(st, "gmi_forward")
    if return_aux:
        return out, den, shift
    return out
