"""FP64 CPU oracle for Gaussian-mixture interpolation (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is a plain, slow, brute-force
O(N*H*W) evaluation of Eq. 1 and Eq. 2 of the paper (section 2) and of their
analytic gradient, written in C (``gmi_oracle.c``) and driven through ctypes.
It shares no code with the CUDA library.

Every function here is pinned by ``tests/test_oracle.py`` against closed forms,
invariants and library routines (see that file's docstring).  Parity status of
each function: forward exact/truncated pinned; backward pinned (finite
differences and torch autograd); pair counts pinned against a k-d tree count;
the per-point, anisotropic and full-covariance extensions (forward_pp,
backward_pp, forward_aniso, backward_aniso, forward_cov, backward_cov) pinned
by their reductions to the simpler forms, closed forms, symmetries, an
independent torch evaluation with autograd and finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gmi_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

EXACT = 0
TRUNCATED = 1


def build(force: bool = False) -> str:
    """Compile ``gmi_oracle.c`` into ``liboracle.so`` (gcc, OpenMP, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            f64p = ctypes.POINTER(ctypes.c_double)
            f32p = ctypes.POINTER(ctypes.c_float)
            i64p = ctypes.POINTER(ctypes.c_int64)
            lib.oracle_forward.argtypes = [f32p, f32p, ctypes.c_int64, ctypes.c_int,
                                           ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                           ctypes.c_int, ctypes.c_double, i64p, ctypes.c_int64,
                                           f64p, f64p, f64p, f64p, i64p]
            lib.oracle_forward.restype = ctypes.c_int
            lib.oracle_backward.argtypes = [f32p, f32p, ctypes.c_int64, ctypes.c_int,
                                            ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                            ctypes.c_int, ctypes.c_double, f32p, f64p, f64p, f64p]
            lib.oracle_backward.restype = ctypes.c_int
            lib.oracle_forward_pp.argtypes = [f32p, f32p, f32p, ctypes.c_int64, ctypes.c_int,
                                              ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                              i64p, ctypes.c_int64, f64p, f64p, f64p, f64p, i64p]
            lib.oracle_forward_pp.restype = ctypes.c_int
            lib.oracle_backward_pp.argtypes = [f32p, f32p, f32p, ctypes.c_int64, ctypes.c_int,
                                               ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                               f32p, f64p, f64p, f64p]
            lib.oracle_backward_pp.restype = ctypes.c_int
            lib.oracle_forward_aniso.argtypes = lib.oracle_forward_pp.argtypes
            lib.oracle_forward_aniso.restype = ctypes.c_int
            lib.oracle_backward_aniso.argtypes = lib.oracle_backward_pp.argtypes
            lib.oracle_backward_aniso.restype = ctypes.c_int
            lib.oracle_forward_cov.argtypes = lib.oracle_forward_pp.argtypes
            lib.oracle_forward_cov.restype = ctypes.c_int
            lib.oracle_backward_cov.argtypes = lib.oracle_backward_pp.argtypes
            lib.oracle_backward_cov.restype = ctypes.c_int
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def forward(points, values, H: int, W: int, sigma: float, mode: int = EXACT,
            k: float = 6.0, pixels=None):
    """Evaluate Eq. 1 / Eq. 2 at ``pixels`` (row-major indices; None = all).

    Returns a dict of float64/int64 arrays: ``image`` ([H,W,C] when pixels is
    None, else [n,C]), ``den``, ``shift``, ``skipped``, ``pairs`` (see
    ``gmi_oracle.c`` for their definitions).
    """
    lib = _load()
    pts = _f32(points).reshape(-1, 2)
    N = pts.shape[0]
    vals = _f32(values)
    C = int(vals.shape[-1]) if vals.ndim == 2 else (int(vals.size // N) if N else 1)
    vals = _f32(vals.reshape(N, C))
    if pixels is None:
        n = H * W
        pix = None
    else:
        pix = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64).ravel())
        n = pix.size
    out = np.empty((n, C), np.float64)
    den = np.empty(n, np.float64)
    shift = np.empty(n, np.float64)
    skipped = np.empty(n, np.float64)
    pairs = np.empty(n, np.int64)
    rc = lib.oracle_forward(_ptr(pts, ctypes.c_float), _ptr(vals, ctypes.c_float), N, C, H, W,
                            float(sigma), int(mode), float(k), _ptr(pix, ctypes.c_int64), n,
                            _ptr(out, ctypes.c_double), _ptr(den, ctypes.c_double),
                            _ptr(shift, ctypes.c_double), _ptr(skipped, ctypes.c_double),
                            _ptr(pairs, ctypes.c_int64))
    if rc != 0:
        raise ValueError("oracle_forward rejected its arguments (rc=%d)" % rc)
    if pixels is None:
        out = out.reshape(H, W, C)
        den = den.reshape(H, W)
        shift = shift.reshape(H, W)
        skipped = skipped.reshape(H, W)
        pairs = pairs.reshape(H, W)
    return {"image": out, "den": den, "shift": shift, "skipped": skipped, "pairs": pairs}


def backward(points, values, H: int, W: int, sigma: float, grad, mode: int = EXACT,
             k: float = 6.0):
    """Analytic gradient of sum(grad * image) w.r.t. points, values, sigma."""
    lib = _load()
    pts = _f32(points).reshape(-1, 2)
    N = pts.shape[0]
    vals = _f32(values).reshape(N, -1)
    C = vals.shape[1]
    g = _f32(grad).reshape(H, W, C)
    gp = np.zeros((N, 2), np.float64)
    gv = np.zeros((N, C), np.float64)
    gs = np.zeros(1, np.float64)
    rc = lib.oracle_backward(_ptr(pts, ctypes.c_float), _ptr(vals, ctypes.c_float), N, C, H, W,
                             float(sigma), int(mode), float(k), _ptr(g, ctypes.c_float),
                             _ptr(gp, ctypes.c_double), _ptr(gv, ctypes.c_double),
                             _ptr(gs, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle_backward rejected its arguments (rc=%d)" % rc)
    return {"points": gp, "values": gv, "sigma": float(gs[0])}


def forward_pp(points, values, sigmas, H: int, W: int, mode: int = EXACT, k: float = 6.0, pixels=None):
    """Eq. 1 / Eq. 2 with a sigma per point (normalisers kept; see
    ``oracle_forward_pp``).  Same outputs as ``forward``; ``shift`` is the
    largest log-weight at the pixel in exact mode."""
    lib = _load()
    pts = _f32(points).reshape(-1, 2)
    N = pts.shape[0]
    vals = _f32(values).reshape(N, -1) if N else _f32(values).reshape(0, np.asarray(values).shape[-1])
    C = int(vals.shape[1])
    sig = _f32(sigmas).reshape(N)
    if pixels is None:
        n = H * W
        pix = None
    else:
        pix = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64).ravel())
        n = pix.size
    out = np.empty((n, C), np.float64)
    den = np.empty(n, np.float64)
    shift = np.empty(n, np.float64)
    skipped = np.empty(n, np.float64)
    pairs = np.empty(n, np.int64)
    rc = lib.oracle_forward_pp(_ptr(pts, ctypes.c_float), _ptr(vals, ctypes.c_float), _ptr(sig, ctypes.c_float),
                               N, C, H, W, int(mode), float(k), _ptr(pix, ctypes.c_int64), n,
                               _ptr(out, ctypes.c_double), _ptr(den, ctypes.c_double),
                               _ptr(shift, ctypes.c_double), _ptr(skipped, ctypes.c_double),
                               _ptr(pairs, ctypes.c_int64))
    if rc != 0:
        raise ValueError("oracle_forward_pp rejected its arguments (rc=%d)" % rc)
    if pixels is None:
        out, den, shift = out.reshape(H, W, C), den.reshape(H, W), shift.reshape(H, W)
        skipped, pairs = skipped.reshape(H, W), pairs.reshape(H, W)
    return {"image": out, "den": den, "shift": shift, "skipped": skipped, "pairs": pairs}


def backward_pp(points, values, sigmas, H: int, W: int, grad, mode: int = EXACT, k: float = 6.0):
    """Analytic gradient of sum(grad * image) w.r.t. points, values and the
    per-point sigmas."""
    lib = _load()
    pts = _f32(points).reshape(-1, 2)
    N = pts.shape[0]
    vals = _f32(values).reshape(N, -1)
    C = vals.shape[1]
    sig = _f32(sigmas).reshape(N)
    g = _f32(grad).reshape(H, W, C)
    gp = np.zeros((N, 2), np.float64)
    gv = np.zeros((N, C), np.float64)
    gs = np.zeros(N, np.float64)
    rc = lib.oracle_backward_pp(_ptr(pts, ctypes.c_float), _ptr(vals, ctypes.c_float), _ptr(sig, ctypes.c_float),
                                N, C, H, W, int(mode), float(k), _ptr(g, ctypes.c_float),
                                _ptr(gp, ctypes.c_double), _ptr(gv, ctypes.c_double), _ptr(gs, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle_backward_pp rejected its arguments (rc=%d)" % rc)
    return {"points": gp, "values": gv, "sigmas": gs}


def forward_aniso(points, values, sigmas_xy, H: int, W: int, mode: int = EXACT, k: float = 6.0, pixels=None):
    """Eq. 1 / Eq. 2 with an axis-aligned covariance diag(sx_i^2, sy_i^2)
    per point (``sigmas_xy[N,2]``, normalisers kept; see
    ``oracle_forward_aniso``).  Same outputs as ``forward_pp``."""
    lib = _load()
    pts = _f32(points).reshape(-1, 2)
    N = pts.shape[0]
    vals = _f32(values).reshape(N, -1) if N else _f32(values).reshape(0, np.asarray(values).shape[-1])
    C = int(vals.shape[1])
    sig = _f32(sigmas_xy).reshape(N, 2)
    if pixels is None:
        n = H * W
        pix = None
    else:
        pix = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64).ravel())
        n = pix.size
    out = np.empty((n, C), np.float64)
    den = np.empty(n, np.float64)
    shift = np.empty(n, np.float64)
    skipped = np.empty(n, np.float64)
    pairs = np.empty(n, np.int64)
    rc = lib.oracle_forward_aniso(_ptr(pts, ctypes.c_float), _ptr(vals, ctypes.c_float),
                                  _ptr(sig, ctypes.c_float), N, C, H, W, int(mode), float(k),
                                  _ptr(pix, ctypes.c_int64), n, _ptr(out, ctypes.c_double),
                                  _ptr(den, ctypes.c_double), _ptr(shift, ctypes.c_double),
                                  _ptr(skipped, ctypes.c_double), _ptr(pairs, ctypes.c_int64))
    if rc != 0:
        raise ValueError("oracle_forward_aniso rejected its arguments (rc=%d)" % rc)
    if pixels is None:
        out, den, shift = out.reshape(H, W, C), den.reshape(H, W), shift.reshape(H, W)
        skipped, pairs = skipped.reshape(H, W), pairs.reshape(H, W)
    return {"image": out, "den": den, "shift": shift, "skipped": skipped, "pairs": pairs}


def backward_aniso(points, values, sigmas_xy, H: int, W: int, grad, mode: int = EXACT, k: float = 6.0):
    """Analytic gradient of sum(grad * image) w.r.t. points, values and the
    per-point (sx, sy)."""
    lib = _load()
    pts = _f32(points).reshape(-1, 2)
    N = pts.shape[0]
    vals = _f32(values).reshape(N, -1)
    C = vals.shape[1]
    sig = _f32(sigmas_xy).reshape(N, 2)
    g = _f32(grad).reshape(H, W, C)
    gp = np.zeros((N, 2), np.float64)
    gv = np.zeros((N, C), np.float64)
    gs = np.zeros((N, 2), np.float64)
    rc = lib.oracle_backward_aniso(_ptr(pts, ctypes.c_float), _ptr(vals, ctypes.c_float),
                                   _ptr(sig, ctypes.c_float), N, C, H, W, int(mode), float(k),
                                   _ptr(g, ctypes.c_float), _ptr(gp, ctypes.c_double), _ptr(gv, ctypes.c_double),
                                   _ptr(gs, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle_backward_aniso rejected its arguments (rc=%d)" % rc)
    return {"points": gp, "values": gv, "sigmas_xy": gs}


def forward_cov(points, values, cov, H: int, W: int, mode: int = EXACT, k: float = 6.0, pixels=None):
    """Eq. 1 / Eq. 2 with a full covariance per point, ``cov[N,3]`` =
    (sx, sy, rho) (see ``oracle_forward_cov``).  Same outputs as
    ``forward_pp``."""
    lib = _load()
    pts = _f32(points).reshape(-1, 2)
    N = pts.shape[0]
    vals = _f32(values).reshape(N, -1) if N else _f32(values).reshape(0, np.asarray(values).shape[-1])
    C = int(vals.shape[1])
    cv = _f32(cov).reshape(N, 3)
    if pixels is None:
        n = H * W
        pix = None
    else:
        pix = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64).ravel())
        n = pix.size
    out = np.empty((n, C), np.float64)
    den = np.empty(n, np.float64)
    shift = np.empty(n, np.float64)
    skipped = np.empty(n, np.float64)
    pairs = np.empty(n, np.int64)
    rc = lib.oracle_forward_cov(_ptr(pts, ctypes.c_float), _ptr(vals, ctypes.c_float), _ptr(cv, ctypes.c_float),
                                N, C, H, W, int(mode), float(k), _ptr(pix, ctypes.c_int64), n,
                                _ptr(out, ctypes.c_double), _ptr(den, ctypes.c_double),
                                _ptr(shift, ctypes.c_double), _ptr(skipped, ctypes.c_double),
                                _ptr(pairs, ctypes.c_int64))
    if rc != 0:
        raise ValueError("oracle_forward_cov rejected its arguments (rc=%d)" % rc)
    if pixels is None:
        out, den, shift = out.reshape(H, W, C), den.reshape(H, W), shift.reshape(H, W)
        skipped, pairs = skipped.reshape(H, W), pairs.reshape(H, W)
    return {"image": out, "den": den, "shift": shift, "skipped": skipped, "pairs": pairs}


def backward_cov(points, values, cov, H: int, W: int, grad, mode: int = EXACT, k: float = 6.0):
    """Analytic gradient of sum(grad * image) w.r.t. points, values and each
    point's (sx, sy, rho)."""
    lib = _load()
    pts = _f32(points).reshape(-1, 2)
    N = pts.shape[0]
    vals = _f32(values).reshape(N, -1)
    C = vals.shape[1]
    cv = _f32(cov).reshape(N, 3)
    g = _f32(grad).reshape(H, W, C)
    gp = np.zeros((N, 2), np.float64)
    gv = np.zeros((N, C), np.float64)
    gc = np.zeros((N, 3), np.float64)
    rc = lib.oracle_backward_cov(_ptr(pts, ctypes.c_float), _ptr(vals, ctypes.c_float), _ptr(cv, ctypes.c_float),
                                 N, C, H, W, int(mode), float(k), _ptr(g, ctypes.c_float),
                                 _ptr(gp, ctypes.c_double), _ptr(gv, ctypes.c_double), _ptr(gc, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle_backward_cov rejected its arguments (rc=%d)" % rc)
    return {"points": gp, "values": gv, "cov": gc}
