"""Autotuner for the forward kernels.

The best micro-tile (4x4, 4x8 or 2x4 pixels per thread) and point-bin edge
depend on sigma (window radius), on the point density and on C.  The tuner
times every candidate on a representative problem with CUDA events (median
of a few runs, after warm-up) and caches the winner per
(GPU name, sigma bucket, density bucket, C) in a JSON file; lookups map a new
problem to its bucket.  Buckets: half-octaves of sigma and octaves of the
point density (points per output pixel).
"""
from __future__ import annotations

import json
import math
import os
import threading

from . import _lib

DEFAULT_VARIANTS = (_lib.VARIANT_MT4x4, _lib.VARIANT_MT4x8, _lib.VARIANT_MT2x4)
DEFAULT_BINS = (0, 1, 2, 4, 8)   # 0 = the library's density rule


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
        """Tuned {"variant", "bin_px"} for the problem's bucket, or None."""
        return self.table.get(self.gpu_name(device), {}).get(bucket(sigma, density, C))

    def save(self):
        d = os.path.dirname(self.path)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = self.path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(self.table, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def tune(self, points, values, sigma: float, H: int, W: int, *, variants=DEFAULT_VARIANTS,
             bins=DEFAULT_BINS, reps: int = 5, warmup: int = 2, save: bool = True):
        """Times every (variant, bin_px) on this problem and records the best
        for its bucket.  Returns (best, {config: median ms})."""
        import torch
        from . import interpolate
        dev = points.device
        out = torch.empty((H, W, values.shape[1]), dtype=torch.float32, device=dev)
        times = {}
        for v in variants:
            for b in bins:
                for _ in range(warmup):
                    interpolate(points, values, sigma, H, W, variant=v, bin_px=b, out=out)
                ms = []
                for _ in range(reps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    interpolate(points, values, sigma, H, W, variant=v, bin_px=b, out=out)
                    e1.record()
                    e1.synchronize()
                    ms.append(e0.elapsed_time(e1))
                ms.sort()
                times[(v, b)] = ms[len(ms) // 2]
        (bv, bb) = min(times, key=times.get)
        best = {"variant": int(bv), "bin_px": int(bb), "ms": times[(bv, bb)]}
        key = bucket(sigma, points.shape[0] / float(H * W), values.shape[1])
        with self._lock:
            self.table.setdefault(self.gpu_name(dev), {})[key] = best
            if save:
                self.save()
        return best, {"%d/%d" % k: t for k, t in times.items()}
