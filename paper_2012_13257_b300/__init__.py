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

__all__ = ["interpolate", "interpolate_backward", "gmi_interpolate", "BatchPlan", "Server", "workspace_size", "GmiError", "MODE_EXACT", "MODE_TRUNCATED", "version", "lib"]


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


def interpolate_backward(points, values, sigma: float, H: int, W: int, image, den, shift, grad_image, *,
                         radius_sigmas: float = 6.0, mode="exact", bin_px: int = 0, variant: int = 0,
                         need=(True, True, True), check: bool = False):
    """Gradients of sum(grad_image * image) w.r.t. points, values and sigma
    (``image``, ``den``, ``shift`` from ``interpolate(..., return_aux=True)``).
    Returns ``(grad_points [N,2], grad_values [N,C], grad_sigma [1])``;
    entries not in ``need`` are None."""
    import torch
    points, values = _check_inputs(points, values)
    N, C = int(points.shape[0]), int(values.shape[1])
    dev = points.device
    for t in (image, den, shift, grad_image):
        if t.device != dev or t.dtype != torch.float32:
            raise ValueError("image, den, shift and grad_image must be float32 on the points' device")
    image, den, shift, grad_image = (t.contiguous() for t in (image, den, shift, grad_image))
    flags = _lib.FLAG_SYNC_CHECK if check else 0
    p = _lib.make_params(sigma, radius_sigmas, _mode(mode), flags, bin_px, variant)
    L = _lib.load()
    nbytes = ctypes.c_size_t(0)
    _lib.check(L.gmi_workspace_size(N, C, int(H), int(W), ctypes.byref(p), ctypes.byref(nbytes)),
               "gmi_workspace_size")
    gp = torch.empty((N, 2), dtype=torch.float32, device=dev) if need[0] else None
    gv = torch.empty((N, C), dtype=torch.float32, device=dev) if need[1] else None
    gs = torch.empty((1,), dtype=torch.float32, device=dev) if need[2] else None
    ws = torch.empty(int(nbytes.value), dtype=torch.uint8, device=dev)
    with torch.cuda.device(dev):
        stream = torch.cuda.current_stream(dev).cuda_stream
        st = L.gmi_backward(points.data_ptr(), values.data_ptr(), N, C, int(H), int(W), ctypes.byref(p),
                            image.data_ptr(), den.data_ptr(), shift.data_ptr(), grad_image.data_ptr(),
                            gp.data_ptr() if gp is not None else None, gv.data_ptr() if gv is not None else None,
                            gs.data_ptr() if gs is not None else None, ws.data_ptr(), int(nbytes.value), stream)
    _lib.check(st, "gmi_backward")
    return gp, gv, gs


def _autograd_function():
    import torch

    class GMIFunction(torch.autograd.Function):
        """Eq. 1 / Eq. 2 as a differentiable op: forward and backward both run
        in libgmi's kernels; the forward saves image, den and shift (the bins
        are rebuilt in the backward)."""

        @staticmethod
        def forward(ctx, points, values, sigma_t, H, W, radius_sigmas, mode, bin_px, variant):
            sigma = float(sigma_t)
            img, den, shift = interpolate(points, values, sigma, H, W, radius_sigmas=radius_sigmas, mode=mode,
                                          bin_px=bin_px, variant=variant, return_aux=True)
            ctx.save_for_backward(points, values, img, den, shift)
            ctx.cfg = (sigma, H, W, radius_sigmas, mode, bin_px, variant, isinstance(sigma_t, torch.Tensor))
            ctx.mark_non_differentiable(den, shift)
            return img, den, shift

        @staticmethod
        def backward(ctx, g, _gden, _gshift):
            points, values, img, den, shift = ctx.saved_tensors
            sigma, H, W, k, mode, bin_px, variant, sig_is_t = ctx.cfg
            need = (ctx.needs_input_grad[0], ctx.needs_input_grad[1], ctx.needs_input_grad[2] and sig_is_t)
            if g is None:
                return (None,) * 9
            gp, gv, gs = interpolate_backward(points, values, sigma, H, W, img, den, shift, g.float(),
                                              radius_sigmas=k, mode=mode, bin_px=bin_px, variant=variant,
                                              need=(need[0], need[1], need[2]))
            gsig = gs.reshape(()) if gs is not None else None
            return gp, gv, gsig, None, None, None, None, None, None

    return GMIFunction


_GMIFunction = None


def gmi_interpolate(points, values, sigma, H: int, W: int, *, radius_sigmas: float = 6.0, mode="exact",
                    bin_px: int = 0, variant: int = 0):
    """Differentiable interpolation (torch.autograd): gradients flow to
    ``points``, ``values`` and, when it is a tensor, ``sigma``.  Returns the
    image [H, W, C]."""
    global _GMIFunction
    if _GMIFunction is None:
        _GMIFunction = _autograd_function()
    img, _, _ = _GMIFunction.apply(points, values, sigma, int(H), int(W), float(radius_sigmas), mode,
                                   int(bin_px), int(variant))
    return img


class BatchPlan:
    """A reusable batched-forward plan (device workspace + pinned staging
    allocated once).  ``forward(images)`` interpolates a list of images, each a
    dict with ``points``, ``values`` (CUDA float32), ``sigma``, ``H``, ``W`` and
    optionally ``out``, ``den``, ``shift``, ``bin_px``, in one batched
    pipeline; with ``use_graph`` the launch sequence is a replayed CUDA graph."""

    def __init__(self, max_images: int, max_points: int, max_pixels: int, C: int = 3, *,
                 radius_sigmas: float = 6.0, mode="exact", variant: int = 0, bin_px: int = 0,
                 check: bool = False):
        p = _lib.make_params(1.0, radius_sigmas, _mode(mode), _lib.FLAG_SYNC_CHECK if check else 0, bin_px, variant)
        h = ctypes.c_void_p()
        _lib.check(_lib.load().gmi_batch_plan_create(int(max_images), int(max_points), int(max_pixels), int(C),
                                                     ctypes.byref(p), ctypes.byref(h)), "gmi_batch_plan_create")
        self._h = h
        self.C = int(C)

    @property
    def nbytes(self) -> int:
        return int(_lib.load().gmi_batch_plan_bytes(self._h))

    def forward(self, images, use_graph: bool = True):
        import torch
        n = len(images)
        descs = (_lib.ImageDesc * max(1, n))()
        outs = []
        keep = []
        dev = None
        for i, im in enumerate(images):
            P, V = _check_inputs(im["points"], im["values"])
            dev = P.device
            H, W = int(im["H"]), int(im["W"])
            out = im.get("out")
            if out is None:
                out = torch.empty((H, W, self.C), dtype=torch.float32, device=dev)
            keep += [P, V]
            d = descs[i]
            d.points, d.values, d.image = P.data_ptr(), V.data_ptr(), out.data_ptr()
            d.den = im["den"].data_ptr() if im.get("den") is not None else None
            d.shift = im["shift"].data_ptr() if im.get("shift") is not None else None
            d.N, d.H, d.W = int(P.shape[0]), H, W
            d.sigma = float(im["sigma"])
            d.bin_px = int(im.get("bin_px", 0))
            outs.append(out)
        stream = torch.cuda.current_stream(dev).cuda_stream if dev is not None else None
        _lib.check(_lib.load().gmi_forward_batched(self._h, descs, n, 1 if use_graph else 0, stream),
                   "gmi_forward_batched")
        self._keep = keep   # inputs stay referenced until the next call
        return outs

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().gmi_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (native threads inside libgmi).

    ``submit(points, values, sigma, H, W, out)`` takes HOST tensors/arrays
    (pinned memory for asynchronous copies; they must stay alive until the
    request completes) and returns a request id; ``wait(id, timeout_ms)``
    returns the latency in seconds once ``out`` holds the image."""

    def __init__(self, budget_bytes: int = 40 << 30, max_batch_images: int = 64,
                 max_batch_pixels: int = 1 << 25, n_streams: int = 2, C: int = 3,
                 radius_sigmas: float = 6.0, mode="exact"):
        L = _lib.load()
        cfg = _lib.ServerConfig()
        L.gmi_server_config_default(ctypes.byref(cfg))
        cfg.budget_bytes = int(budget_bytes)
        cfg.max_batch_images = int(max_batch_images)
        cfg.max_batch_pixels = int(max_batch_pixels)
        cfg.n_streams = int(n_streams)
        cfg.C = int(C)
        cfg.radius_sigmas = float(radius_sigmas)
        cfg.mode = _mode(mode)
        h = ctypes.c_void_p()
        _lib.check(L.gmi_server_create(ctypes.byref(cfg), ctypes.byref(h)), "gmi_server_create")
        self._h = h
        self.C = int(C)
        self._keep = {}

    @staticmethod
    def _ptr(a):
        import numpy as np
        if hasattr(a, "data_ptr"):
            if a.device.type != "cpu" or not a.is_contiguous() or a.dtype.__str__() != "torch.float32":
                raise ValueError("server buffers must be contiguous float32 host tensors")
            return a.data_ptr()
        a = np.ascontiguousarray(a)
        if a.dtype != np.float32:
            raise ValueError("server buffers must be float32")
        return a.ctypes.data

    def submit(self, points, values, sigma: float, H: int, W: int, out) -> int:
        rid = ctypes.c_uint64(0)
        n = int(points.shape[0])
        _lib.check(_lib.load().gmi_server_submit(self._h, self._ptr(points) if n else None,
                                                 self._ptr(values) if n else None, n, int(H), int(W),
                                                 float(sigma), self._ptr(out), ctypes.byref(rid)),
                   "gmi_server_submit")
        self._keep[rid.value] = (points, values, out)
        return int(rid.value)

    def wait(self, rid: int, timeout_ms: int = -1) -> float:
        lat = ctypes.c_double(0.0)
        st = _lib.load().gmi_server_wait(self._h, int(rid), int(timeout_ms), ctypes.byref(lat))
        if st != 6:   # finished (or unknown): its buffers may be released
            self._keep.pop(int(rid), None)
        _lib.check(st, "gmi_server_wait")
        return float(lat.value)

    def poll(self, rid: int) -> bool:
        st = _lib.load().gmi_server_poll(self._h, int(rid))
        if st == 6:
            return False
        _lib.check(st, "gmi_server_poll")
        return True

    def stats(self):
        c, l, p = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        b = ctypes.c_size_t()
        _lib.check(_lib.load().gmi_server_stats(self._h, ctypes.byref(c), ctypes.byref(l), ctypes.byref(p),
                                                ctypes.byref(b)), "gmi_server_stats")
        return {"completed": c.value, "launches": l.value, "pixels": p.value, "bytes_in_use": b.value}

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().gmi_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
