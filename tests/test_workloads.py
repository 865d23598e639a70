"""Host checks of the seeded input generators that the sweeps rely on (no GPU)."""
import numpy as np

import workloads as wl


def test_reconstruction_case_geometry():
    """Low-resolution samples sit at the centres of the f x f blocks; for an
    odd factor that centre is a full-resolution pixel centre, so the truth
    there equals the sample exactly."""
    f, side = 3, 48
    pts, vals, low, truth = wl.reconstruction_case(f, side)
    n = side // f
    assert low.shape == (n, n, 3) and truth.shape == (side, side, 3)
    assert np.array_equal(pts[n + 2], np.float32([(2 + 0.5) * f, (1 + 0.5) * f]))
    assert np.array_equal(truth[1::f, 1::f], low)
    assert np.array_equal(vals.reshape(n, n, 3), low)
    assert truth.min() >= 0.0 and truth.max() <= 1.0


def test_field_refactor_keeps_the_upsampling_values():
    """smooth_field is field_params + eval_field with the same draws."""
    rng1, rng2 = np.random.default_rng(11), np.random.default_rng(11)
    xy = rng1.uniform(0, 64, (100, 2)).astype(np.float32)
    rng2.uniform(0, 64, (100, 2))
    a = wl.smooth_field(rng1, xy, 3, 64.0)
    b = wl.eval_field(wl.field_params(rng2, 3), xy, 64.0)
    assert np.array_equal(a, b)
