"""Autotuner for the forward kernels.

The best micro-tile (4x4, 4x8 or 2x4 pixels per thread), point-bin edge and
points per stage depend on sigma (window radius), on the point density and on
C.  Points per stage is the near-field gather's staging: "staged" copies each
warp's candidate window, up to 352 records (224 for 8-pixel micro-tiles), into
shared memory before its threads walk it; "direct" stages nothing and every
thread loads its candidates through L1.  (The staging buffer itself is the
largest that keeps the register-limited 16 warps per SM resident; larger
buffers measured slower everywhere, so it is not a tuning axis.)  The
library's gmi_autotune times every (micro-tile, bin edge) on a representative
problem with CUDA events (median of a few runs after a warm-up), once per
staging choice; this class keeps the winner per (GPU name, sigma bucket,
density bucket, C) in a JSON file, and lookups map a new problem to its
bucket.  Buckets: half-octaves of sigma and octaves of the point density
(points per output pixel).
"""
from __future__ import annotations

import json
import math
import os
import threading

from . import _lib

DEFAULT_VARIANTS = (_lib.VARIANT_MT4x4, _lib.VARIANT_MT4x8, _lib.VARIANT_MT2x4)
DEFAULT_BINS = (0, 1, 2, 4, 8)   # 0 = the library's density rule
DEFAULT_GATHERS = ("staged", "direct")
_GATHER_CODES = {"staged": _lib.GATHER_STAGED, "direct": _lib.GATHER_DIRECT}


def _default_path():
    return os.environ.get("GMI_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "gmi_autotune.json"))


def bucket(sigma: float, density: float, C: int):
    s = round(math.log2(max(float(sigma), 1e-6)) * 2) / 2
    d = round(math.log2(max(float(density), 1e-9)))
    return "s%+.1f_d%+d_c%d" % (s, d, int(C))


class Autotuner:
    def __init__(self, path: str | None = None):
        self.path = path or _default_path()
        self._lock = threading.Lock()
        self.table = {}
        if os.path.exists(self.path):
            try:
                with open(self.path) as f:
                    self.table = json.load(f)
            except (OSError, ValueError):
                self.table = {}

    @staticmethod
    def gpu_name(device=None) -> str:
        import torch
        return torch.cuda.get_device_name(device)

    def lookup(self, sigma: float, density: float, C: int, device=None):
        """Tuned {"variant", "bin_px", "gather", "ms"} for the problem's bucket,
        or None."""
        return self.table.get(self.gpu_name(device), {}).get(bucket(sigma, density, C))

    def save(self):
        d = os.path.dirname(self.path)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = self.path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(self.table, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def tune(self, points, values, sigma: float, H: int, W: int, *, bins=DEFAULT_BINS,
             gathers=DEFAULT_GATHERS, reps: int = 5, save: bool = True, **_):
        """Times every (variant, bin_px) on this problem (gmi_autotune), once
        per staging choice in ``gathers``, and records the best for its bucket.
        Returns (best, {"variant/bin/gather": ms})."""
        import ctypes
        import torch
        from . import _check_inputs, _mode, _stream_handle
        points, values = _check_inputs(points, values)
        dev = points.device
        N, C = int(points.shape[0]), int(values.shape[1])
        nb = len(bins)
        barr = (ctypes.c_int * nb)(*[int(b) for b in bins])
        table = {}
        for gname in gathers:
            p = _lib.make_params(float(sigma))
            p.gather = _GATHER_CODES[gname]
            best = _lib.Params()
            times = (ctypes.c_float * (3 * nb))()
            with torch.cuda.device(dev):
                _lib.check(_lib.load().gmi_autotune(points.data_ptr(), values.data_ptr(), N, C, int(H), int(W),
                                                    ctypes.byref(p), barr, nb, int(reps), ctypes.byref(best),
                                                    times, _stream_handle(dev)), "gmi_autotune")
            for vi, v in enumerate(DEFAULT_VARIANTS):
                for k, b in enumerate(bins):
                    table["%d/%d/%s" % (v, b, gname)] = float(times[vi * nb + k])
        key_best = min(table, key=table.get)
        v, b, gname = key_best.split("/")
        res = {"variant": int(v), "bin_px": int(b), "gather": gname, "ms": table[key_best]}
        key = bucket(sigma, N / float(H * W), C)
        with self._lock:
            self.table.setdefault(self.gpu_name(dev), {})[key] = res
            if save:
                self.save()
        return res, table
