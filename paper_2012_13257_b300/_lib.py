"""ctypes declarations of the libgmi C ABI (``include/gmi.h``).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libgmi.so``.  Loading fails loudly when the library has not been
built; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# GMI_CHECKED=1 in the environment loads the checked build (bounds checks
# that record instead of trapping, guard areas after workspace regions)
CHECKED = os.environ.get("GMI_CHECKED", "") not in ("", "0")
LIB_PATH = os.path.join(HERE, "libgmi_checked.so" if CHECKED else "libgmi.so")

GMI_OK = 0
STATUS_NAMES = {
    0: "GMI_OK", 1: "GMI_ERR_INVALID_ARG", 2: "GMI_ERR_NONFINITE", 3: "GMI_ERR_WORKSPACE",
    4: "GMI_ERR_CUDA", 5: "GMI_ERR_BUDGET", 6: "GMI_ERR_TIMEOUT", 7: "GMI_ERR_UNSUPPORTED",
    8: "GMI_ERR_NOT_FOUND", 9: "GMI_ERR_CAPACITY", 10: "GMI_ERR_INTERNAL",
}
MODE_EXACT = 0
MODE_TRUNCATED = 1
FLAG_SYNC_CHECK = 0x1
FLAG_GRAPH = 0x2
VARIANT_AUTO, VARIANT_MT4x4, VARIANT_MT4x8, VARIANT_MT2x4, VARIANT_MT4x2 = 0, 1, 2, 3, 4
GATHER_AUTO, GATHER_STAGED, GATHER_DIRECT = 0, 1, 2
# default params.gather of the calls this process makes (gmi.set_gather; interpolate and
# BatchPlan also take a per-call choice)
DEFAULT_GATHER = GATHER_AUTO
STAGES = ("bin", "near", "far", "backward")
NOALLOC_SCRATCH_BYTES = 32 << 20   # GMI_NOALLOC_SCRATCH_BYTES


class GmiError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        super().__init__("%s%s" % (where + ": " if where else "",
                                   STATUS_NAMES.get(self.status, "status %d" % status)))


class Params(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_float), ("radius_sigmas", ctypes.c_float), ("mode", ctypes.c_int),
                ("flags", ctypes.c_uint), ("bin_px", ctypes.c_int), ("variant", ctypes.c_int),
                ("gather", ctypes.c_int), ("reserved", ctypes.c_int)]


class WsLayout(ctypes.Structure):
    _fields_ = [("off", ctypes.c_size_t), ("oob", ctypes.c_size_t), ("sxy", ctypes.c_size_t),
                ("sval", ctypes.c_size_t), ("perm", ctypes.c_size_t), ("bin_px", ctypes.c_int),
                ("nbx", ctypes.c_int), ("nby", ctypes.c_int), ("total", ctypes.c_size_t),
                ("ubound", ctypes.c_size_t), ("mth", ctypes.c_int), ("mtw", ctypes.c_int),
                ("wtx", ctypes.c_int), ("wty", ctypes.c_int), ("sat", ctypes.c_size_t)]


class ImageDesc(ctypes.Structure):
    _fields_ = [("points", ctypes.c_void_p), ("values", ctypes.c_void_p), ("image", ctypes.c_void_p),
                ("den", ctypes.c_void_p), ("shift", ctypes.c_void_p), ("N", ctypes.c_int64),
                ("H", ctypes.c_int), ("W", ctypes.c_int), ("sigma", ctypes.c_float), ("bin_px", ctypes.c_int)]


class GradDesc(ctypes.Structure):
    _fields_ = [("points", ctypes.c_void_p), ("values", ctypes.c_void_p), ("image", ctypes.c_void_p),
                ("den", ctypes.c_void_p), ("shift", ctypes.c_void_p), ("grad_image", ctypes.c_void_p),
                ("grad_points", ctypes.c_void_p), ("grad_values", ctypes.c_void_p), ("grad_sigma", ctypes.c_void_p),
                ("N", ctypes.c_int64), ("H", ctypes.c_int), ("W", ctypes.c_int), ("sigma", ctypes.c_float),
                ("bin_px", ctypes.c_int)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("max_batch_images", ctypes.c_int),
                ("max_batch_pixels", ctypes.c_int64), ("n_streams", ctypes.c_int), ("C", ctypes.c_int),
                ("radius_sigmas", ctypes.c_float), ("mode", ctypes.c_int), ("reserved", ctypes.c_int)]


class ServerCounters(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("launches", ctypes.c_uint64), ("pixels", ctypes.c_uint64),
                ("bytes_in_use", ctypes.c_size_t), ("in_flight", ctypes.c_int), ("max_in_flight", ctypes.c_int),
                ("reserved", ctypes.c_uint64 * 4)]


# name -> (restype, argtypes), mirroring include/gmi.h
_vp, _i64, _int, _f, _sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_size_t
_u64p = ctypes.POINTER(ctypes.c_uint64)
SIGNATURES = {
    "gmi_version": (ctypes.c_char_p, []),
    "gmi_status_string": (ctypes.c_char_p, [_int]),
    "gmi_params_default": (_int, [ctypes.POINTER(Params)]),
    "gmi_workspace_size": (_int, [_i64, _int, _int, _int, ctypes.POINTER(Params), ctypes.POINTER(_sz)]),
    "gmi_forward": (_int, [_vp, _vp, _i64, _int, _int, _int, ctypes.POINTER(Params), _vp, _vp, _vp,
                           _vp, _sz, _vp]),
    "gmi_backward": (_int, [_vp, _vp, _i64, _int, _int, _int, ctypes.POINTER(Params), _vp, _vp, _vp, _vp,
                            _vp, _vp, _vp, _vp, _sz, _vp]),
    "gmi_forward_pp": (_int, [_vp, _vp, _vp, _i64, _int, _int, _int, ctypes.POINTER(Params), _vp, _vp,
                              _vp, _sz, _vp]),
    "gmi_backward_pp": (_int, [_vp, _vp, _vp, _i64, _int, _int, _int, ctypes.POINTER(Params), _vp, _vp,
                               _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "gmi_forward_aniso": (_int, [_vp, _vp, _vp, _i64, _int, _int, _int, ctypes.POINTER(Params), _vp, _vp,
                                 _vp, _sz, _vp]),
    "gmi_backward_aniso": (_int, [_vp, _vp, _vp, _i64, _int, _int, _int, ctypes.POINTER(Params), _vp, _vp,
                                  _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "gmi_forward_cov": (_int, [_vp, _vp, _vp, _i64, _int, _int, _int, ctypes.POINTER(Params), _vp, _vp,
                               _vp, _sz, _vp]),
    "gmi_backward_cov": (_int, [_vp, _vp, _vp, _i64, _int, _int, _int, ctypes.POINTER(Params), _vp, _vp,
                                _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "gmi_workspace_status": (_int, [_vp, _vp]),
    "gmi_check_workspace": (_int, [_i64, _int, _int, _int, ctypes.POINTER(Params), _vp, ctypes.c_size_t, _vp,
                                   ctypes.POINTER(ctypes.c_uint32)]),
    "gmi_batch_check_workspace": (_int, [_vp, _vp, ctypes.POINTER(ctypes.c_uint32)]),
    "gmi_is_checked_build": (_int, []),
    "gmi_workspace_layout": (_int, [_i64, _int, _int, _int, ctypes.POINTER(Params), ctypes.POINTER(WsLayout)]),
    "gmi_forward_noalloc": (_int, [_vp, _vp, _i64, _int, _int, _int, ctypes.POINTER(Params), _vp, _vp, _vp,
                                   _vp]),
    "gmi_forward_host_workspace_size": (_int, [_i64, _int, _int, _int, ctypes.POINTER(Params),
                                               ctypes.POINTER(_sz)]),
    "gmi_forward_host": (_int, [_vp, _vp, _i64, _int, _int, _int, ctypes.POINTER(Params), _vp, _vp, _sz, _vp]),
    "gmi_profile_enable": (_int, [_int]),
    "gmi_profile_read": (_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), _int]),
    "gmi_measure_unit_rates": (_int, [ctypes.POINTER(ctypes.c_double)]),
    "gmi_set_wait_polls": (_int, [_i64]),
    "gmi_autotune": (_int, [_vp, _vp, ctypes.c_int64, _int, _int, _int, ctypes.POINTER(Params),
                            ctypes.POINTER(_int), _int, _int, ctypes.POINTER(Params),
                            ctypes.POINTER(ctypes.c_float), _vp]),
    "gmi_batch_plan_create": (_int, [_int, _i64, _i64, _int, ctypes.POINTER(Params), ctypes.POINTER(_vp)]),
    "gmi_batch_plan_destroy": (_int, [_vp]),
    "gmi_batch_plan_bytes": (_sz, [_vp]),
    "gmi_forward_batched": (_int, [_vp, ctypes.POINTER(ImageDesc), _int, _int, _vp]),
    "gmi_backward_batched": (_int, [_vp, ctypes.POINTER(GradDesc), _int, _vp]),
    "gmi_forward_stacked": (_int, [_vp, _vp, _vp, _int, _i64, _int, _int, ctypes.POINTER(_f), _vp, _vp, _vp, _int,
                                   _vp]),
    "gmi_backward_stacked": (_int, [_vp, _vp, _vp, _int, _i64, _int, _int, ctypes.POINTER(_f), _vp, _vp, _vp, _vp,
                                    _vp, _vp, _vp, _vp]),
    "gmi_server_config_default": (_int, [ctypes.POINTER(ServerConfig)]),
    "gmi_server_create": (_int, [ctypes.POINTER(ServerConfig), ctypes.POINTER(_vp)]),
    "gmi_server_submit": (_int, [_vp, _vp, _vp, _i64, _int, _int, _f, _vp, _u64p]),
    "gmi_server_submit_device": (_int, [_vp, _vp, _vp, _i64, _int, _int, _f, _vp, _u64p]),
    "gmi_server_get_counters": (_int, [_vp, ctypes.POINTER(ServerCounters)]),
    "gmi_server_set_log": (_int, [_vp, ctypes.c_char_p]),
    "gmi_server_wait": (_int, [_vp, ctypes.c_uint64, _int, ctypes.POINTER(ctypes.c_double)]),
    "gmi_server_poll": (_int, [_vp, ctypes.c_uint64]),
    "gmi_server_stats": (_int, [_vp, _u64p, _u64p, _u64p, ctypes.POINTER(_sz)]),
    "gmi_server_destroy": (_int, [_vp]),
}

_lib = None


def load():
    """Loads libgmi.so (raising if it has not been built) and declares its ABI."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(os.path.basename(LIB_PATH) + " is not built (run paper_2012_13257_b300/build.py or "
                              "__graft_entry__.build()); there is no non-CUDA fallback")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(status: int, where: str = ""):
    if status != GMI_OK:
        raise GmiError(status, where)


def make_params(sigma: float, radius_sigmas: float = 6.0, mode: int = MODE_EXACT, flags: int = 0,
                bin_px: int = 0, variant: int = 0) -> Params:
    p = Params()
    load().gmi_params_default(ctypes.byref(p))
    p.sigma = float(sigma)
    p.radius_sigmas = float(radius_sigmas)
    p.mode = int(mode)
    p.flags = int(flags)
    p.bin_px = int(bin_px)
    p.variant = int(variant)
    p.gather = int(DEFAULT_GATHER)
    return p
