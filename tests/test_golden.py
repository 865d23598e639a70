"""Stored expected values (tests/golden/oracle_cases.txt, written by
tests/golden/make_golden.py from the FP64 oracle alone).

CPU: the oracle as it stands still reproduces them (any later change to its
arithmetic shows here), and the two-point case matches its closed form, a
logistic sigmoid of (d1^2 - d2^2) / (2 sigma^2) (Eq. 1 with two terms).
GPU: the CUDA path reproduces them within the forward tolerance."""
import math
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
TOL_FWD = 1e-4


def load_cases():
    cases, cur = [], None
    for line in open(os.path.join(HERE, "golden", "oracle_cases.txt")):
        if line.startswith("#") or not line.strip():
            continue
        key, _, rest = line.rstrip("\n").partition(" ")
        if key == "case":
            cur = {"name": rest}
            cases.append(cur)
        elif key == "cite":
            cur["cite"] = rest
        elif key == "shape":
            H, W, C, mode, k = rest.split()
            cur.update(H=int(H), W=int(W), C=int(C), mode=int(mode), k=float(k))
        else:
            cur[key] = np.array([float(v) for v in rest.split()])
    for c in cases:
        c["points"] = c["points"].astype(np.float32).reshape(-1, 2)
        c["values"] = c["values"].astype(np.float32).reshape(-1, c["C"])
        c["image"] = c["image"].reshape(c["H"], c["W"], c["C"])
        c["den"] = c["den"].reshape(c["H"], c["W"])
    return cases


CASES = load_cases()


def run_oracle(c):
    if "sigmas" in c:
        return oracle.forward_pp(c["points"], c["values"], c["sigmas"].astype(np.float32), c["H"], c["W"],
                                 mode=c["mode"], k=c["k"])
    return oracle.forward(c["points"], c["values"], c["H"], c["W"], float(c["sigma"][0]), mode=c["mode"], k=c["k"])


def test_fixture_file_is_complete():
    names = [c["name"] for c in CASES]
    assert names == ["two_points_exact", "random12_exact", "random12_truncated", "random12_per_point_truncated"]
    for c in CASES:
        assert c["cite"].startswith("Eq. 1")


@pytest.mark.parametrize("case", CASES, ids=lambda c: c["name"])
def test_oracle_reproduces_the_stored_values(case):
    ref = run_oracle(case)
    np.testing.assert_allclose(ref["image"], case["image"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(ref["den"], case["den"], rtol=1e-13, atol=0)


def test_two_point_fixture_is_the_closed_form():
    c = CASES[0]
    s = float(c["sigma"][0])
    p = c["points"].astype(np.float64)
    yy, xx = np.meshgrid(np.arange(c["H"]) + 0.5, np.arange(c["W"]) + 0.5, indexing="ij")
    d1 = (xx - p[0, 0]) ** 2 + (yy - p[0, 1]) ** 2
    d2 = (xx - p[1, 0]) ** 2 + (yy - p[1, 1]) ** 2
    t = 1.0 / (1.0 + np.exp(-(d1 - d2) / (2 * s * s)))   # weight of the second point
    want = c["values"][0][None, None, :] * (1 - t)[..., None] + c["values"][1][None, None, :] * t[..., None]
    np.testing.assert_allclose(c["image"], want, rtol=0, atol=1e-13)
    m = np.minimum(d1, d2)   # exact mode keeps den relative to the nearest point
    np.testing.assert_allclose(c["den"], np.exp(-(d1 - m) / (2 * s * s)) + np.exp(-(d2 - m) / (2 * s * s)),
                               rtol=1e-13)
    assert math.isclose(float(c["image"][0, 0, 0]), float(want[0, 0, 0]), rel_tol=1e-13)


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES, ids=lambda c: c["name"])
def test_cuda_path_reproduces_the_stored_values(cuda_device, case):
    import torch
    import paper_2012_13257_b300 as gmi
    from gpu_helpers import to_dev
    P, V = to_dev(case["points"], cuda_device), to_dev(case["values"], cuda_device)
    mode = "truncated" if case["mode"] == oracle.TRUNCATED else "exact"
    if "sigmas" in case:
        sig = case["sigmas"].astype(np.float32)
        out = gmi.interpolate_pp(P, V, to_dev(sig, cuda_device), float(sig.max()), case["H"], case["W"],
                                 radius_sigmas=case["k"], check=True, mode="truncated")
    else:
        out = gmi.interpolate(P, V, float(case["sigma"][0]), case["H"], case["W"], mode=mode,
                              radius_sigmas=case["k"], check=True)
    torch.cuda.synchronize()
    decided = run_oracle(case)["skipped"] < 1e-3
    err = np.abs(out.cpu().numpy().astype(np.float64) - case["image"])[decided]
    assert err.max() <= TOL_FWD, err.max()
