"""Shared helpers of the GPU parity tests (comparison against the oracle)."""
import numpy as np
from scipy.spatial import cKDTree

# Forward tolerance: max-abs error on colours in [0, 1].
TOL_FWD = 1e-4


def to_dev(a, device):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device=device)


def sample_pixels(points, H, W, n_random=2048, n_border=512, n_tiles=4, tile=8, n_far=256, seed=0):
    """Pixel subset for full-size parity: random pixels, border pixels, whole
    tiles and the pixels farthest from any point (far field)."""
    rng = np.random.default_rng(seed)
    sel = [rng.integers(0, H * W, n_random)]
    border = np.concatenate([np.arange(W), (H - 1) * W + np.arange(W),
                             np.arange(H) * W, np.arange(H) * W + W - 1])
    sel.append(rng.choice(border, min(n_border, border.size), replace=False))
    for _ in range(n_tiles):
        ty, tx = rng.integers(0, max(1, H - tile)), rng.integers(0, max(1, W - tile))
        yy, xx = np.meshgrid(np.arange(ty, min(H, ty + tile)), np.arange(tx, min(W, tx + tile)), indexing="ij")
        sel.append((yy * W + xx).ravel())
    if n_far and points.shape[0]:
        yy, xx = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
        q = np.stack([xx.ravel(), yy.ravel()], 1)
        d, _ = cKDTree(points.astype(np.float64)).query(q, workers=-1)
        sel.append(np.argsort(-d)[:n_far])
    return np.unique(np.concatenate(sel)).astype(np.int64)


def log_scaled_den(den, shift, sigma):
    """log of the unshifted density sum, from a (den, shift) pair."""
    return np.log(np.asarray(den, np.float64)) - np.asarray(shift, np.float64) / (2.0 * sigma * sigma)
