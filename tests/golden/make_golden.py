"""Writes the stored expected values under tests/golden/ from the FP64 oracle
(and nothing else): small fixed cases of Eq. 1 / Eq. 2 (section 2), exact and
truncated, shared and per-point sigma, each with its inputs written out in
full so that the fixture stands on its own.

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def cases():
    """(name, citation, points, values, sigma or per-point sigmas, H, W, mode, k)."""
    rng = np.random.default_rng(20121325)
    out = []
    # two points: the colour is a logistic sigmoid of (d1^2 - d2^2) / (2 sigma^2)
    out.append(("two_points_exact", "Eq. 1, Eq. 2 (section 2): two known points, exact sums",
                np.float32([[1.25, 2.5], [5.75, 3.0]]), np.float32([[1.0, 0.0, 0.25], [0.0, 1.0, 0.75]]),
                0.9, 5, 7, oracle.EXACT, 6.0))
    # a small random case, exact and truncated
    pts = np.stack([rng.uniform(-1, 9, 12), rng.uniform(-1, 7, 12)], 1).astype(np.float32)
    vals = rng.uniform(0, 1, (12, 3)).astype(np.float32)
    out.append(("random12_exact", "Eq. 1, Eq. 2 (section 2): 12 points, exact sums", pts, vals, 0.8, 6, 8,
                oracle.EXACT, 6.0))
    out.append(("random12_truncated", "Eq. 1, Eq. 2 (section 2): 12 points, radius k sigma (reading of 'close "
                "enough')", pts, vals, 0.8, 6, 8, oracle.TRUNCATED, 2.0))
    sig = rng.uniform(0.5, 1.2, 12).astype(np.float32)
    out.append(("random12_per_point_truncated", "Eq. 1, Eq. 2 with a sigma per point (normalisers kept), "
                "radius k sigma_i", pts, vals, sig, 6, 8, oracle.TRUNCATED, 2.5))
    return out


def fmt(a):
    return " ".join("%.17g" % float(v) for v in np.asarray(a, np.float64).ravel())


def main():
    path = os.path.join(HERE, "oracle_cases.txt")
    with open(path, "w") as f:
        f.write("# Expected values of small cases, written by tests/golden/make_golden.py from the FP64 oracle.\n")
        f.write("# Each case: name, citation, H W C mode k, points (x y per point), values, sigma(s), then\n")
        f.write("# the image row-major [H,W,C] and den [H,W].\n")
        for name, cite, pts, vals, sig, H, W, mode, k in cases():
            if np.ndim(sig) == 0:
                ref = oracle.forward(pts, vals, H, W, float(sig), mode=mode, k=k)
                sig_line = "sigma %.17g" % float(sig)
            else:
                ref = oracle.forward_pp(pts, vals, sig, H, W, mode=mode, k=k)
                sig_line = "sigmas " + fmt(sig)
            f.write("case %s\n" % name)
            f.write("cite %s\n" % cite)
            f.write("shape %d %d %d %d %.17g\n" % (H, W, vals.shape[1], mode, k))
            f.write("points " + fmt(pts) + "\n")
            f.write("values " + fmt(vals) + "\n")
            f.write(sig_line + "\n")
            f.write("image " + fmt(ref["image"]) + "\n")
            f.write("den " + fmt(ref["den"]) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
