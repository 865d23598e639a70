"""Builds libgmi.so (all CUDA sources of the package) in-tree with nvcc for sm_103a."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libgmi.so")
OUT_CHECKED = os.path.join(HERE, "libgmi_checked.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _stale(obj, src, headers):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(f) > t for f in [src] + headers)


def build(force: bool = False, verbose: bool = False, extra=(), checked: bool = False) -> str:
    """Builds libgmi.so, or with ``checked`` libgmi_checked.so: the same
    sources compiled with -DGMI_CHECKED (bounds checks that record instead of
    trapping, guard areas after every workspace region)."""
    nvcc = os.environ.get("NVCC", "nvcc")
    out_path = OUT_CHECKED if checked else OUT
    build_dir = BUILD + ("_checked" if checked else "")
    if checked:
        extra = tuple(extra) + ("-DGMI_CHECKED",)
    os.makedirs(build_dir, exist_ok=True)
    headers = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))
    objs = []
    procs = []
    for src in sources():
        obj = os.path.join(build_dir, os.path.basename(src) + ".o")
        objs.append(obj)
        if force or _stale(obj, src, headers):
            cmd = [nvcc] + ARCH + FLAGS + list(extra) + ["-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd), flush=True)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stdout.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError("nvcc failed on: " + ", ".join(failed))
    if force or procs or not os.path.exists(out_path):
        tmp = out_path + ".tmp%d" % os.getpid()
        subprocess.check_call([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart", "-lpthread"])
        os.replace(tmp, out_path)
    return out_path


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="--ptxas" in sys.argv or "-v" in sys.argv,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [], checked="--checked" in sys.argv)
