"""The checked build (libgmi_checked.so: every queue, slot and sorted-array
index tested before use, guard areas after every workspace region) run over
the forward (dense, ragged, far field, split tiles, truncated, both gathers,
every micro-tile, graph replay), backward, per-point (isotropic and full
covariance, exact and truncated) and batched paths: no bounds check fails,
every guard is intact, and the results still match the FP64 oracle.  It runs
in a child process (GMI_CHECKED=1 selects the checked library at load)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_checked_build_paths_clean(cuda_device):
    lib = os.path.join(ROOT, "paper_2012_13257_b300", "libgmi_checked.so")
    if not os.path.exists(lib):
        sys.path.insert(0, ROOT)
        from paper_2012_13257_b300 import build as b
        b.build(checked=True)
    env = dict(os.environ, GMI_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_calls.py")], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0 and "ALL OK" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
