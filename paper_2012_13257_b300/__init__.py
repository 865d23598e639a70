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

__all__ = ["set_gather", "release_workspaces", "interpolate", "interpolate_host", "interpolate_backward", "gmi_interpolate", "interpolate_pp",
           "interpolate_backward_pp", "gmi_interpolate_pp", "BatchPlan", "gmi_interpolate_batch", "gmi_interpolate_stacked", "Server", "workspace_size", "GmiError", "MODE_EXACT", "MODE_TRUNCATED", "version", "lib"]


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


_param_cache = {}
_ws_size_cache = {}
_table_cache = {}
_offset_cache = {}


def _stream_handle(dev):
    """Raw handle of the current CUDA stream of `dev` (a cheap query where
    torch offers one)."""
    import torch
    raw = getattr(torch._C, "_cuda_getCurrentRawStream", None)
    if raw is not None:
        return raw(dev.index if dev.index is not None else torch.cuda.current_device())
    return torch.cuda.current_stream(dev).cuda_stream
_ws_buffers = {}


def set_gather(kind: str) -> None:
    """Chooses how the near-field gather reads its candidates, for every later
    call of this process: "auto" (the default: staged for one shared sigma),
    "staged" (each warp stages its window in shared memory) or "direct"
    (each thread loads its candidates through the L1 cache).  Both give the
    same sums; the choice exists to compare their speed."""
    if kind not in _GATHERS:
        raise ValueError("gather must be one of %s" % sorted(_GATHERS))
    _lib.DEFAULT_GATHER = _GATHERS[kind]


_GATHERS = {"auto": _lib.GATHER_AUTO, "staged": _lib.GATHER_STAGED, "direct": _lib.GATHER_DIRECT}


def _gather_code(gather) -> int:
    """params.gather for a call: the process default (set_gather) when None,
    else "auto", "staged" or "direct"."""
    if gather is None:
        return int(_lib.DEFAULT_GATHER)
    if gather not in _GATHERS:
        raise ValueError("gather must be one of %s" % sorted(_GATHERS))
    return _GATHERS[gather]


def _params(sigma, radius_sigmas, mode, flags, bin_px, variant, gather=None):
    g = _gather_code(gather)
    key = (float(sigma), float(radius_sigmas), mode, flags, bin_px, variant, g)
    p = _param_cache.get(key)
    if p is None:
        if len(_param_cache) > 4096:
            _param_cache.clear()
        p = _lib.make_params(sigma, radius_sigmas, mode, flags, bin_px, variant)
        p.gather = g
        _param_cache[key] = p
    return p


def _ws_bytes(N, C, H, W, p, key):
    n = _ws_size_cache.get(key)
    if n is None:
        c = ctypes.c_size_t(0)
        _lib.check(_lib.load().gmi_workspace_size(N, C, H, W, ctypes.byref(p), ctypes.byref(c)), "gmi_workspace_size")
        if len(_ws_size_cache) > 4096:
            _ws_size_cache.clear()
        n = _ws_size_cache[key] = int(c.value)
    return n


def _workspace(dev, stream, nbytes):
    """Scratch reused per (device, stream): calls on one stream run in order,
    so consecutive calls may share it; other streams get their own."""
    import torch
    key = (dev.index, stream)
    buf = _ws_buffers.get(key)
    if buf is None or buf.numel() < nbytes:
        buf = torch.empty(max(nbytes, 1 << 20), dtype=torch.uint8, device=dev)
        _ws_buffers[key] = buf
    return buf


def release_workspaces():
    """Drops the cached per-stream scratch buffers."""
    _ws_buffers.clear()


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
                check: bool = False, graph: bool = False, out=None, gather=None):
    """Forward pass of Eq. 1 / Eq. 2 onto an H x W raster.

    Returns the image ``[H, W, C]``; with ``return_aux`` also the per-pixel
    ``den`` and ``shift`` planes (den = sum_i exp(-(d_i^2 - shift)/(2 sigma^2))).
    ``check=True`` synchronises and raises on device-detected errors
    (non-finite inputs).  ``graph=True`` replays a cached CUDA graph of the
    launch sequence when the same tensors (``out`` included) and sizes come
    again: pass ``out`` to reuse buffers across calls.  Runs on the current
    CUDA stream.  ``gather`` ("staged", "direct" or "auto"; None: the
    process default of set_gather) chooses how the near-field gather reads
    its candidates, e.g. as the autotuner picked it.
    """
    import torch
    points, values = _check_inputs(points, values)
    N, C = int(points.shape[0]), int(values.shape[1])
    H, W = int(H), int(W)
    dev = points.device
    flags = (_lib.FLAG_SYNC_CHECK if check else 0) | (_lib.FLAG_GRAPH if graph else 0)
    md = _mode(mode)
    p = _params(sigma, radius_sigmas, md, flags, bin_px, variant, gather)
    nbytes = _ws_bytes(N, C, H, W, p, (N, C, H, W, float(sigma), float(radius_sigmas), md, bin_px, variant))
    if out is None:
        out = torch.empty((H, W, C), dtype=torch.float32, device=dev)
    den = torch.empty((H, W), dtype=torch.float32, device=dev) if return_aux else None
    shift = torch.empty((H, W), dtype=torch.float32, device=dev) if return_aux else None
    stream = _stream_handle(dev)
    ws = _workspace(dev, stream, nbytes)
    if torch.cuda.current_device() != dev.index:
        with torch.cuda.device(dev):
            return interpolate(points, values, sigma, H, W, radius_sigmas=radius_sigmas, mode=mode,
                               bin_px=bin_px, variant=variant, return_aux=return_aux, check=check,
                               graph=graph, out=out, gather=gather)
    st = _lib.load().gmi_forward(points.data_ptr(), values.data_ptr(), N, C, H, W, ctypes.byref(p),
                                 out.data_ptr(), den.data_ptr() if den is not None else None,
                                 shift.data_ptr() if shift is not None else None, ws.data_ptr(),
                                 ws.numel(), stream)
    _lib.check(st, "gmi_forward")
    if return_aux:
        return out, den, shift
    return out


_host_ws_size_cache = {}


def interpolate_host(points, values, sigma: float, H: int, W: int, *, radius_sigmas: float = 6.0,
                     mode="exact", bin_px: int = 0, variant: int = 0, check: bool = False,
                     graph: bool = False, out=None, device=None):
    """Eq. 1 / Eq. 2 end to end from host memory (``gmi_forward_host``):
    ``points [N, 2]`` and ``values [N, C]`` are CPU float32 tensors (pinned
    for asynchronous copies), the image comes back in ``out`` (a CPU float32
    tensor ``[H, W, C]``, allocated pinned when not given).  The uploads, the
    kernels and the download run in order on the current CUDA stream of
    ``device`` (default: the current device); synchronise that stream before
    reading ``out``, or pass ``check=True``.  ``graph=True`` replays the copies
    and the kernels as one cached CUDA graph for the same buffers."""
    import torch
    if not (isinstance(points, torch.Tensor) and isinstance(values, torch.Tensor)):
        raise TypeError("points and values must be torch tensors")
    if points.device.type != "cpu" or values.device.type != "cpu":
        raise ValueError("points and values must be host (CPU) tensors")
    if points.dtype != torch.float32 or values.dtype != torch.float32:
        raise TypeError("points and values must be float32")
    if points.dim() != 2 or points.shape[1] != 2 or values.dim() != 2 or values.shape[0] != points.shape[0]:
        raise ValueError("points must have shape [N, 2] and values [N, C]")
    points, values = points.contiguous(), values.contiguous()
    N, C = int(points.shape[0]), int(values.shape[1])
    H, W = int(H), int(W)
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index)
    flags = (_lib.FLAG_SYNC_CHECK if check else 0) | (_lib.FLAG_GRAPH if graph else 0)
    md = _mode(mode)
    p = _params(sigma, radius_sigmas, md, flags, bin_px, variant)
    key = (N, C, H, W, float(sigma), float(radius_sigmas), md, bin_px, variant)
    nbytes = _host_ws_size_cache.get(key)
    if nbytes is None:
        c = ctypes.c_size_t(0)
        _lib.check(_lib.load().gmi_forward_host_workspace_size(N, C, H, W, ctypes.byref(p), ctypes.byref(c)),
                   "gmi_forward_host_workspace_size")
        nbytes = _host_ws_size_cache[key] = int(c.value)
    if out is None:
        out = torch.empty((H, W, C), dtype=torch.float32).pin_memory()
    elif out.device.type != "cpu" or out.dtype != torch.float32 or tuple(out.shape) != (H, W, C) \
            or not out.is_contiguous():
        raise ValueError("out must be a contiguous CPU float32 tensor of shape [H, W, C]")
    with torch.cuda.device(dev):
        stream = _stream_handle(dev)
        ws = _workspace(dev, stream, nbytes)
        st = _lib.load().gmi_forward_host(points.data_ptr(), values.data_ptr(), N, C, H, W, ctypes.byref(p),
                                          out.data_ptr(), ws.data_ptr(), ws.numel(), stream)
    _lib.check(st, "gmi_forward_host")
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
    H, W = int(H), int(W)
    flags = _lib.FLAG_SYNC_CHECK if check else 0
    md = _mode(mode)
    p = _params(sigma, radius_sigmas, md, flags, bin_px, variant)
    nbytes = _ws_bytes(N, C, H, W, p, (N, C, H, W, float(sigma), float(radius_sigmas), md, bin_px, variant))
    gp = torch.empty((N, 2), dtype=torch.float32, device=dev) if need[0] else None
    gv = torch.empty((N, C), dtype=torch.float32, device=dev) if need[1] else None
    gs = torch.empty((1,), dtype=torch.float32, device=dev) if need[2] else None
    stream = _stream_handle(dev)
    ws = _workspace(dev, stream, nbytes)
    if torch.cuda.current_device() != dev.index:
        with torch.cuda.device(dev):
            return interpolate_backward(points, values, sigma, H, W, image, den, shift, grad_image,
                                        radius_sigmas=radius_sigmas, mode=mode, bin_px=bin_px, variant=variant,
                                        need=need, check=check)
    st = _lib.load().gmi_backward(points.data_ptr(), values.data_ptr(), N, C, H, W, ctypes.byref(p),
                                  image.data_ptr(), den.data_ptr(), shift.data_ptr(), grad_image.data_ptr(),
                                  gp.data_ptr() if gp is not None else None,
                                  gv.data_ptr() if gv is not None else None,
                                  gs.data_ptr() if gs is not None else None, ws.data_ptr(), ws.numel(), stream)
    _lib.check(st, "gmi_backward")
    return gp, gv, gs


_sigma_cache = {}


def _cached_host_copy(t, read):
    """read(t) for a CUDA tensor, cached per (tensor object, version): reading
    device memory synchronises, so an unchanged sigma tensor is read once and
    one updated in place (an optimizer step) is read again.  The entry holds a
    weak reference to the very tensor, so a new tensor that reuses a freed
    address or object id never sees another tensor's values."""
    import weakref
    e = _sigma_cache.get(id(t))
    if e is not None and e[0]() is t and e[1] == t._version:
        return e[2]
    v = read(t)
    if len(_sigma_cache) > 4096:
        _sigma_cache.clear()
    _sigma_cache[id(t)] = (weakref.ref(t), t._version, v)
    return v


def _sigma_value(sigma_t) -> float:
    """Host value of sigma (a float, or a CPU or CUDA scalar tensor)."""
    import torch
    if not isinstance(sigma_t, torch.Tensor):
        return float(sigma_t)
    if sigma_t.device.type == "cpu":
        return float(sigma_t)
    return _cached_host_copy(sigma_t, lambda t: float(t))


def _autograd_function():
    import torch

    class GMIFunction(torch.autograd.Function):
        """Eq. 1 / Eq. 2 as a differentiable op: forward and backward both run
        in libgmi's kernels; the forward keeps image, den and shift for the
        backward (the bins are rebuilt there)."""

        @staticmethod
        def forward(ctx, points, values, sigma_t, H, W, radius_sigmas, mode, bin_px, variant):
            sigma = _sigma_value(sigma_t)
            img, den, shift = interpolate(points, values, sigma, H, W, radius_sigmas=radius_sigmas, mode=mode,
                                          bin_px=bin_px, variant=variant, return_aux=True)
            ctx.set_materialize_grads(False)
            # tensors (the output included) go through save_for_backward: kept
            # on ctx directly, the output would form a reference cycle with its
            # grad_fn and outlive the step until Python's cycle collector ran
            ctx.save_for_backward(points, values, img, den, shift)
            ctx.cfg = (sigma, H, W, radius_sigmas, mode, bin_px, variant, isinstance(sigma_t, torch.Tensor))
            return img

        @staticmethod
        def backward(ctx, g):
            if g is None:
                return (None,) * 9
            points, values, img, den, shift = ctx.saved_tensors
            sigma, H, W, k, mode, bin_px, variant, sig_is_t = ctx.cfg
            need = (ctx.needs_input_grad[0], ctx.needs_input_grad[1], ctx.needs_input_grad[2] and sig_is_t)
            gp, gv, gs = interpolate_backward(points.detach(), values.detach(), sigma, H, W, img, den, shift,
                                              g.float(), radius_sigmas=k, mode=mode, bin_px=bin_px,
                                              variant=variant, need=need)
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
    return _GMIFunction.apply(points, values, sigma, int(H), int(W), float(radius_sigmas), mode,
                              int(bin_px), int(variant))


def _check_sigmas(sigmas, points):
    """(contiguous sigmas, floats per point): [N] isotropic, [N,2] = (sx, sy),
    [N,3] = (sx, sy, rho)."""
    import torch
    if not isinstance(sigmas, torch.Tensor) or sigmas.dtype != torch.float32 or sigmas.device != points.device:
        raise TypeError("sigmas must be a float32 tensor on the points' device")
    N = points.shape[0]
    if sigmas.dim() == 2 and sigmas.shape[0] == N and sigmas.shape[1] in (2, 3):
        return sigmas.contiguous(), int(sigmas.shape[1])
    if sigmas.dim() == 1 and sigmas.shape[0] == N:
        return sigmas.contiguous(), 1
    raise ValueError("sigmas must have shape [N] (isotropic), [N, 2] (sx, sy) or [N, 3] (sx, sy, rho)")


_PP_CALLS = {1: ("gmi_forward_pp", "gmi_backward_pp"), 2: ("gmi_forward_aniso", "gmi_backward_aniso"),
             3: ("gmi_forward_cov", "gmi_backward_cov")}


def interpolate_pp(points, values, sigmas, sigma_bound: float, H: int, W: int, *, radius_sigmas: float = 6.0,
                   mode="exact", bin_px: int = 0, variant: int = 0, return_aux: bool = False, check: bool = False,
                   graph: bool = False, out=None):
    """Forward pass with a sigma per point, normalisers kept: over all points
    (``mode="exact"``, weights relative to each pixel's largest; points below
    exp(-radius_sigmas^2/2) of it may be left out) or inside each point's
    ``radius_sigmas``-sigma disc or ellipse (``mode="truncated"``).  ``sigmas`` is
    ``[N]`` (isotropic sigma_i), ``[N, 2]`` (axis-aligned (sx_i, sy_i)) or
    ``[N, 3]`` (a full covariance (sx_i, sy_i, rho_i), |rho_i| <= 0.99).
    ``sigma_bound`` must bound every sigma from above (it sets the search
    radius; a tight bound is faster); for a full covariance it bounds the
    square root of each covariance's largest eigenvalue.  With ``return_aux`` also returns
    ``den``: in truncated mode sum_i sigma_bound^2 / (sx_i sy_i) exp(-(dx^2/sx_i^2 +
    dy^2/sy_i^2)/2) (full covariance: sigma_bound^2 / sqrt(det S_i)
    exp(-d^T S_i^-1 d / 2)); in exact mode the weights' sum relative to the
    pixel's largest weight (>= 1).  ``check=True`` synchronises and raises on out-of-range
    or non-finite sigmas (and the other device-detected errors)."""
    import torch
    points, values = _check_inputs(points, values)
    sigmas, kind = _check_sigmas(sigmas, points)
    N, C = int(points.shape[0]), int(values.shape[1])
    H, W = int(H), int(W)
    dev = points.device
    flags = (_lib.FLAG_SYNC_CHECK if check else 0) | (_lib.FLAG_GRAPH if graph else 0)
    md = _mode(mode)
    p = _params(sigma_bound, radius_sigmas, md, flags, bin_px, variant)
    nbytes = _ws_bytes(N, C, H, W, p, (N, C, H, W, float(sigma_bound), float(radius_sigmas), md, bin_px, variant))
    if out is None:
        out = torch.empty((H, W, C), dtype=torch.float32, device=dev)
    den = torch.empty((H, W), dtype=torch.float32, device=dev) if return_aux else None
    if torch.cuda.current_device() != dev.index:
        with torch.cuda.device(dev):
            return interpolate_pp(points, values, sigmas, sigma_bound, H, W, radius_sigmas=radius_sigmas,
                                  mode=mode, bin_px=bin_px, variant=variant, return_aux=return_aux, check=check,
                                  graph=graph, out=out)
    stream = _stream_handle(dev)
    ws = _workspace(dev, stream, nbytes)
    name = _PP_CALLS[kind][0]
    st = getattr(_lib.load(), name)(points.data_ptr(), values.data_ptr(), sigmas.data_ptr(), N, C, H, W,
                                    ctypes.byref(p), out.data_ptr(), den.data_ptr() if den is not None else None,
                                    ws.data_ptr(), ws.numel(), stream)
    _lib.check(st, name)
    if return_aux:
        return out, den
    return out


def interpolate_backward_pp(points, values, sigmas, sigma_bound: float, H: int, W: int, image, den, grad_image, *,
                            radius_sigmas: float = 6.0, mode="exact", bin_px: int = 0, variant: int = 0,
                            need=(True, True, True), check: bool = False):
    """Gradients of sum(grad_image * image) w.r.t. points, values and the
    per-point sigmas (``image``, ``den`` from ``interpolate_pp(...,
    return_aux=True)``).  Returns ``(grad_points [N,2], grad_values [N,C],
    grad_sigmas)``, the last shaped like ``sigmas``; entries not in ``need``
    are None."""
    import torch
    points, values = _check_inputs(points, values)
    sigmas, kind = _check_sigmas(sigmas, points)
    N, C = int(points.shape[0]), int(values.shape[1])
    dev = points.device
    for t in (image, den, grad_image):
        if t.device != dev or t.dtype != torch.float32:
            raise ValueError("image, den and grad_image must be float32 on the points' device")
    image, den, grad_image = (t.contiguous() for t in (image, den, grad_image))
    H, W = int(H), int(W)
    flags = _lib.FLAG_SYNC_CHECK if check else 0
    md = _mode(mode)
    p = _params(sigma_bound, radius_sigmas, md, flags, bin_px, variant)
    nbytes = _ws_bytes(N, C, H, W, p, (N, C, H, W, float(sigma_bound), float(radius_sigmas), md, bin_px, variant))
    gp = torch.empty((N, 2), dtype=torch.float32, device=dev) if need[0] else None
    gv = torch.empty((N, C), dtype=torch.float32, device=dev) if need[1] else None
    gs = torch.empty(tuple(sigmas.shape), dtype=torch.float32, device=dev) if need[2] else None
    if torch.cuda.current_device() != dev.index:
        with torch.cuda.device(dev):
            return interpolate_backward_pp(points, values, sigmas, sigma_bound, H, W, image, den, grad_image,
                                           radius_sigmas=radius_sigmas, mode=mode, bin_px=bin_px, variant=variant,
                                           need=need, check=check)
    stream = _stream_handle(dev)
    ws = _workspace(dev, stream, nbytes)
    name = _PP_CALLS[kind][1]
    st = getattr(_lib.load(), name)(points.data_ptr(), values.data_ptr(), sigmas.data_ptr(), N, C, H, W,
                                    ctypes.byref(p), image.data_ptr(), den.data_ptr(), grad_image.data_ptr(),
                                    gp.data_ptr() if gp is not None else None,
                                    gv.data_ptr() if gv is not None else None,
                                    gs.data_ptr() if gs is not None else None, ws.data_ptr(), ws.numel(), stream)
    _lib.check(st, name)
    return gp, gv, gs


def _pp_function():
    import torch

    class GMIPPFunction(torch.autograd.Function):
        """Per-point-sigma interpolation as a differentiable op; forward and
        backward run in libgmi's kernels."""

        @staticmethod
        def forward(ctx, points, values, sigmas, sigma_bound, H, W, radius_sigmas, mode, bin_px, variant):
            img, den = interpolate_pp(points, values, sigmas, sigma_bound, H, W, radius_sigmas=radius_sigmas,
                                      mode=mode, bin_px=bin_px, variant=variant, return_aux=True)
            ctx.set_materialize_grads(False)
            ctx.save_for_backward(points, values, sigmas, img, den)
            ctx.cfg = (sigma_bound, H, W, radius_sigmas, mode, bin_px, variant)
            return img

        @staticmethod
        def backward(ctx, g):
            if g is None:
                return (None,) * 10
            points, values, sigmas, img, den = ctx.saved_tensors
            bound, H, W, k, mode, bin_px, variant = ctx.cfg
            need = tuple(ctx.needs_input_grad[:3])
            gp, gv, gs = interpolate_backward_pp(points.detach(), values.detach(), sigmas.detach(), bound, H, W,
                                                 img, den, g.float(), radius_sigmas=k, mode=mode, bin_px=bin_px,
                                                 variant=variant, need=need)
            if gs is not None:
                gs = gs.reshape(sigmas.shape)
            return gp, gv, gs, None, None, None, None, None, None, None

    return GMIPPFunction


_GMIPPFunction = None


def gmi_interpolate_pp(points, values, sigmas, sigma_bound: float, H: int, W: int, *, radius_sigmas: float = 6.0,
                       mode="exact", bin_px: int = 0, variant: int = 0):
    """Differentiable per-point-sigma interpolation (over all points, or
    truncated inside each point's ``radius_sigmas``-sigma disc or ellipse
    with ``mode="truncated"``): gradients flow to ``points``, ``values`` and
    ``sigmas`` ([N] isotropic, [N, 2] axis-aligned (sx, sy) or [N, 3] full
    (sx, sy, rho)).  ``sigma_bound`` >= every sigma.  Returns [H, W, C]."""
    global _GMIPPFunction
    if _GMIPPFunction is None:
        _GMIPPFunction = _pp_function()
    return _GMIPPFunction.apply(points, values, sigmas, float(sigma_bound), int(H), int(W), float(radius_sigmas),
                                _mode(mode), int(bin_px), int(variant))


def _flat_views(shapes, dev, dtype=None):
    """One allocation for several tensors: views of the given shapes, each
    starting on a 16-byte boundary (so the kernels may use vector stores)."""
    import math
    import torch
    sizes = [int(math.prod(sh)) for sh in shapes]
    offs, o = [], 0
    for n in sizes:
        offs.append(o)
        o += (n + 3) // 4 * 4
    buf = torch.empty(max(o, 1), dtype=dtype or torch.float32, device=dev)
    return [buf[a:a + n].view(sh) for a, n, sh in zip(offs, sizes, shapes)]


def _np_table(ctype, n):
    """numpy structured array laid out exactly like the ctypes Structure."""
    import numpy as np
    fields = ctype._fields_
    names = [f[0] for f in fields]
    fmt = {ctypes.c_void_p: np.uint64, ctypes.c_int64: np.int64, ctypes.c_int: np.int32, ctypes.c_float: np.float32}
    dt = np.dtype({"names": names, "formats": [fmt[f[1]] for f in fields],
                   "offsets": [getattr(ctype, nm).offset for nm in names], "itemsize": ctypes.sizeof(ctype)})
    return np.zeros(max(n, 1), dtype=dt)


def _scratch_table(ctype, n):
    """A zeroed table reused across calls (the batched C calls copy their
    table into the plan's staging before returning, so it is free again)."""
    key = (ctype, n)
    t = _table_cache.get(key)
    if t is None:
        t = _table_cache[key] = _np_table(ctype, n)
    else:
        t.fill(0)
    return t


def _ptrs(t, B):
    """Addresses of the B equal slices t[0], ..., t[B-1] of a contiguous tensor."""
    import numpy as np
    step = t[0].numel() * t.element_size() if B else 0
    key = (B, step)
    off = _offset_cache.get(key)
    if off is None:
        if len(_offset_cache) > 1024:
            _offset_cache.clear()
        off = _offset_cache[key] = np.arange(B, dtype=np.uint64) * np.uint64(step)
    return off + np.uint64(t.data_ptr())


class BatchPlan:
    """A reusable batched-forward plan (device workspace + pinned staging
    allocated once).  ``forward(images)`` interpolates a list of images, each a
    dict with ``points``, ``values`` (CUDA float32), ``sigma``, ``H``, ``W`` and
    optionally ``out``, ``den``, ``shift``, ``bin_px``, in one batched
    pipeline; with ``use_graph`` the launch sequence is a replayed CUDA graph."""

    def __init__(self, max_images: int, max_points: int, max_pixels: int, C: int = 3, *,
                 radius_sigmas: float = 6.0, mode="exact", variant: int = 0, bin_px: int = 0,
                 check: bool = False, gather=None):
        p = _lib.make_params(1.0, radius_sigmas, _mode(mode), _lib.FLAG_SYNC_CHECK if check else 0, bin_px, variant)
        p.gather = _gather_code(gather)
        h = ctypes.c_void_p()
        _lib.check(_lib.load().gmi_batch_plan_create(int(max_images), int(max_points), int(max_pixels), int(C),
                                                     ctypes.byref(p), ctypes.byref(h)), "gmi_batch_plan_create")
        self._h = h
        self.C = int(C)

    @property
    def nbytes(self) -> int:
        return int(_lib.load().gmi_batch_plan_bytes(self._h))

    def forward(self, images, use_graph: bool = True):
        import numpy as np
        import torch
        n = len(images)
        tab = _np_table(_lib.ImageDesc, n)
        dev = images[0]["points"].device if n else None
        need_out = [i for i, im in enumerate(images) if im.get("out") is None]
        fresh = _flat_views([(int(images[i]["H"]), int(images[i]["W"]), self.C) for i in need_out], dev) \
            if need_out else []
        outs = [im.get("out") for im in images]
        for i, v in zip(need_out, fresh):
            outs[i] = v
        keep = []
        for i, im in enumerate(images):
            P, V = _check_inputs(im["points"], im["values"])
            keep += [P, V]
            tab["points"][i], tab["values"][i], tab["image"][i] = P.data_ptr(), V.data_ptr(), outs[i].data_ptr()
            if im.get("den") is not None:
                tab["den"][i] = im["den"].data_ptr()
            if im.get("shift") is not None:
                tab["shift"][i] = im["shift"].data_ptr()
            tab["N"][i] = P.shape[0]
            tab["H"][i], tab["W"][i] = int(im["H"]), int(im["W"])
            tab["sigma"][i] = float(im["sigma"])
            tab["bin_px"][i] = int(im.get("bin_px", 0))
        stream = _stream_handle(dev) if dev is not None else None
        _lib.check(_lib.load().gmi_forward_batched(
            self._h, ctypes.cast(tab.ctypes.data, ctypes.POINTER(_lib.ImageDesc)), n, 1 if use_graph else 0,
            stream), "gmi_forward_batched")
        self._keep = (keep, tab)   # inputs stay referenced until the next call
        return outs

    def forward_table(self, tab, n: int, stream, use_graph: bool = True):
        """Launch from a prebuilt numpy ImageDesc table (see _np_table)."""
        _lib.check(_lib.load().gmi_forward_batched(
            self._h, ctypes.cast(tab.ctypes.data, ctypes.POINTER(_lib.ImageDesc)), int(n), 1 if use_graph else 0,
            stream), "gmi_forward_batched")

    def backward_table(self, tab, n: int, stream):
        """Launch the batched backward from a prebuilt numpy GradDesc table."""
        _lib.check(_lib.load().gmi_backward_batched(
            self._h, ctypes.cast(tab.ctypes.data, ctypes.POINTER(_lib.GradDesc)), int(n), stream),
            "gmi_backward_batched")

    def backward(self, images):
        """Batched backward.  Each entry: ``points``, ``values``, ``sigma``,
        ``H``, ``W``, ``image``, ``den``, ``shift`` (forward outputs),
        ``grad`` (upstream [H,W,C]) and optionally ``bin_px`` and ``need``
        (points, values, sigma).  Returns a list of (grad_points, grad_values,
        grad_sigma) tuples (None where not needed)."""
        import torch
        n = len(images)
        tab = _np_table(_lib.GradDesc, n)
        dev = images[0]["points"].device if n else None
        needs = [im.get("need", (True, True, True)) for im in images]
        Ns = [int(im["points"].shape[0]) for im in images]
        Cs = [int(im["values"].shape[1]) for im in images]
        gps = iter(_flat_views([(N, 2) for N, nd in zip(Ns, needs) if nd[0]], dev))
        gvs = iter(_flat_views([(N, C) for N, C, nd in zip(Ns, Cs, needs) if nd[1]], dev))
        gss = iter(_flat_views([(1,) for nd in needs if nd[2]], dev))
        res, keep = [], []
        for i, im in enumerate(images):
            P, V = _check_inputs(im["points"], im["values"])
            nd = needs[i]
            gp = next(gps) if nd[0] else None
            gv = next(gvs) if nd[1] else None
            gs = next(gss) if nd[2] else None
            img, den, shift = im["image"].contiguous(), im["den"].contiguous(), im["shift"].contiguous()
            g = im["grad"].contiguous().float()
            keep += [P, V, img, den, shift, g]
            tab["points"][i], tab["values"][i] = P.data_ptr(), V.data_ptr()
            tab["image"][i], tab["den"][i] = img.data_ptr(), den.data_ptr()
            tab["shift"][i], tab["grad_image"][i] = shift.data_ptr(), g.data_ptr()
            if gp is not None:
                tab["grad_points"][i] = gp.data_ptr()
            if gv is not None:
                tab["grad_values"][i] = gv.data_ptr()
            if gs is not None:
                tab["grad_sigma"][i] = gs.data_ptr()
            tab["N"][i] = Ns[i]
            tab["H"][i], tab["W"][i] = int(im["H"]), int(im["W"])
            tab["sigma"][i] = float(im["sigma"])
            tab["bin_px"][i] = int(im.get("bin_px", 0))
            res.append((gp, gv, gs))
        stream = _stream_handle(dev) if dev is not None else None
        _lib.check(_lib.load().gmi_backward_batched(
            self._h, ctypes.cast(tab.ctypes.data, ctypes.POINTER(_lib.GradDesc)), n, stream), "gmi_backward_batched")
        self._keep_bwd = (keep, tab)
        return res

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

    def submit_device(self, points, values, sigma: float, H: int, W: int, out) -> int:
        """Submits a request whose tensors live on the server's CUDA device:
        no copies, the image is written into ``out`` in place.  The tensors
        must stay alive, and the inputs unchanged, until the request
        completes."""
        import torch
        for t in (points, values, out):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous() and t.dtype == torch.float32):
                raise ValueError("device requests take contiguous float32 CUDA tensors")
        rid = ctypes.c_uint64(0)
        n = int(points.shape[0])
        _lib.check(_lib.load().gmi_server_submit_device(self._h, points.data_ptr() if n else None,
                                                        values.data_ptr() if n else None, n, int(H), int(W),
                                                        float(sigma), out.data_ptr(), ctypes.byref(rid)),
                   "gmi_server_submit_device")
        self._keep[rid.value] = (points, values, out)
        return int(rid.value)

    def counters(self):
        c = _lib.ServerCounters()
        _lib.check(_lib.load().gmi_server_get_counters(self._h, ctypes.byref(c)), "gmi_server_get_counters")
        return {"completed": c.completed, "launches": c.launches, "pixels": c.pixels,
                "bytes_in_use": c.bytes_in_use, "in_flight": c.in_flight, "max_in_flight": c.max_in_flight}

    def set_log(self, path):
        """One JSON line per completed request (submit, admit, launch and done
        times in seconds since the server started) to ``path``; None stops."""
        _lib.check(_lib.load().gmi_server_set_log(self._h, path.encode() if path else None), "gmi_server_set_log")

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


def _batch_function():
    import torch

    class GMIBatchFunction(torch.autograd.Function):
        """B images through one batched forward (CUDA-graph replay) and one
        batched backward.  Inputs are flattened: points_0, values_0, sigma_0,
        points_1, ...; returns the B images."""

        @staticmethod
        def forward(ctx, plan, sizes, *flat):
            B = len(sizes)
            dev = flat[0].device
            aux = _flat_views([(H, W) for H, W in sizes] * 2, dev)
            ims = []
            for b in range(B):
                P, V, S = flat[3 * b], flat[3 * b + 1], flat[3 * b + 2]
                H, W = sizes[b]
                ims.append({"points": P, "values": V, "sigma": _sigma_value(S), "H": H, "W": W,
                            "den": aux[b], "shift": aux[B + b]})
            outs = plan.forward(ims, use_graph=True)
            ctx.set_materialize_grads(False)
            # every tensor through save_for_backward (no reference cycle with
            # the outputs); the rest as plain values
            saved = []
            for b in range(B):
                saved += [flat[3 * b], flat[3 * b + 1], outs[b], aux[b], aux[B + b]]
            ctx.save_for_backward(*saved)
            ctx.plan = plan
            ctx.meta = [(ims[b]["sigma"], ims[b]["H"], ims[b]["W"]) for b in range(B)]
            ctx.sig_t = [isinstance(flat[3 * b + 2], torch.Tensor) for b in range(B)]
            return tuple(outs)

        @staticmethod
        def backward(ctx, *grads):
            sv = ctx.saved_tensors
            req = []
            for b, g in enumerate(grads):
                P, V, img, den, shift = sv[5 * b:5 * b + 5]
                sigma, H, W = ctx.meta[b]
                if g is None:
                    g = torch.zeros_like(img)
                need = (ctx.needs_input_grad[2 + 3 * b], ctx.needs_input_grad[3 + 3 * b],
                        ctx.needs_input_grad[4 + 3 * b] and ctx.sig_t[b])
                req.append({"points": P.detach(), "values": V.detach(), "sigma": sigma, "H": H, "W": W,
                            "image": img, "den": den, "shift": shift, "grad": g, "need": need})
            res = ctx.plan.backward(req)
            out = [None, None]
            for gp, gv, gs in res:
                out += [gp, gv, gs.reshape(()) if gs is not None else None]
            return tuple(out)

    return GMIBatchFunction


_GMIBatchFunction = None


def gmi_interpolate_batch(plan, points, values, sigmas, sizes):
    """Differentiable batched interpolation on a BatchPlan: lists of points
    [N_b,2], values [N_b,C], sigmas (floats or 0-d tensors) and sizes (H, W);
    returns the list of images.  The whole batch is one forward launch (graph
    replay) and one batched backward."""
    global _GMIBatchFunction
    if _GMIBatchFunction is None:
        _GMIBatchFunction = _batch_function()
    flat = []
    for P, V, S in zip(points, values, sigmas):
        flat += [P, V, S]
    return list(_GMIBatchFunction.apply(plan, [tuple(map(int, hw)) for hw in sizes], *flat))


def _stacked_function():
    import numpy as np
    import torch

    fptr = ctypes.POINTER(ctypes.c_float)

    class GMIStackedFunction(torch.autograd.Function):
        """B equal-shaped images ([B,N,2] points, [B,N,C] values, [B] sigmas)
        through one batched forward and one batched backward
        (gmi_forward_stacked / gmi_backward_stacked: the per-image
        descriptors are built in the library from the stacked tensors'
        addresses, so the host work does not grow with B)."""

        @staticmethod
        def forward(ctx, plan, H, W, points, values, sigmas):
            B, N = int(points.shape[0]), int(points.shape[1])
            C = int(values.shape[2])
            dev = points.device
            points, values = points.contiguous(), values.contiguous()
            sig = np.ascontiguousarray(_sigma_list(sigmas, B), dtype=np.float32)
            out = torch.empty((B, H, W, C), dtype=torch.float32, device=dev)
            den = torch.empty((B, H, W), dtype=torch.float32, device=dev)
            shift = torch.empty((B, H, W), dtype=torch.float32, device=dev)
            _lib.check(_lib.load().gmi_forward_stacked(
                plan._h, points.data_ptr(), values.data_ptr(), B, N, H, W, sig.ctypes.data_as(fptr),
                out.data_ptr(), den.data_ptr(), shift.data_ptr(), 1, _stream_handle(dev)), "gmi_forward_stacked")
            ctx.set_materialize_grads(False)
            # tensors (the output included) through save_for_backward: no
            # reference cycle between the output and its grad_fn
            ctx.plan = plan
            ctx.save_for_backward(points, values, out, den, shift)
            ctx.aux = (sig, H, W, isinstance(sigmas, torch.Tensor))
            return out

        @staticmethod
        def backward(ctx, g):
            if g is None:
                return (None,) * 6
            points, values, out, den, shift = ctx.saved_tensors
            sig, H, W, sig_t = ctx.aux
            B, N, C = int(points.shape[0]), int(points.shape[1]), int(values.shape[2])
            dev = points.device
            g = g.contiguous().float()
            need = ctx.needs_input_grad
            gp = torch.empty((B, N, 2), dtype=torch.float32, device=dev) if need[3] else None
            gv = torch.empty((B, N, C), dtype=torch.float32, device=dev) if need[4] else None
            gs = torch.empty((B,), dtype=torch.float32, device=dev) if (need[5] and sig_t) else None
            _lib.check(_lib.load().gmi_backward_stacked(
                ctx.plan._h, points.data_ptr(), values.data_ptr(), B, N, H, W, sig.ctypes.data_as(fptr),
                out.data_ptr(), den.data_ptr(), shift.data_ptr(), g.data_ptr(),
                gp.data_ptr() if gp is not None else None, gv.data_ptr() if gv is not None else None,
                gs.data_ptr() if gs is not None else None, _stream_handle(dev)), "gmi_backward_stacked")
            return (None, None, None, gp, gv, gs)

    return GMIStackedFunction


def _sigma_list(sigmas, B):
    import numpy as np
    import torch
    if isinstance(sigmas, torch.Tensor):
        if sigmas.device.type != "cpu":
            return _cached_host_copy(sigmas, lambda t: t.detach().float().cpu().numpy().reshape(B))
        return sigmas.detach().float().numpy().reshape(B)
    return np.broadcast_to(np.asarray(sigmas, dtype=np.float32), (B,))


_GMIStackedFunction = None


def gmi_interpolate_stacked(plan, points, values, sigmas, H: int, W: int):
    """Differentiable batched interpolation of B equal-shaped images:
    points [B,N,2], values [B,N,C], sigmas [B] (tensor: differentiable) ->
    images [B,H,W,C], one batched forward and one batched backward."""
    global _GMIStackedFunction
    if _GMIStackedFunction is None:
        _GMIStackedFunction = _stacked_function()
    return _GMIStackedFunction.apply(plan, int(H), int(W), points, values, sigmas)


def measure_unit_rates(device=None) -> dict:
    """Measured results per SM per clock of the units the near-field gather
    is bound by on this GPU: ``ex2`` (SFU), ``ffma`` and ``ffma2`` (FP32 FMA
    pipe, scalar and packed).  Synchronous, a few milliseconds."""
    import torch
    r = (ctypes.c_double * 3)()
    with torch.cuda.device(device if device is not None else torch.cuda.current_device()):
        _lib.check(_lib.load().gmi_measure_unit_rates(r), "gmi_measure_unit_rates")
    return {"ex2": r[0], "ffma": r[1], "ffma2": r[2]}
