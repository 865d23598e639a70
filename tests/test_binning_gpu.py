"""The binning step (bin keys, counts, exclusive scan, scatter) checked bit
for bit: after gmi_forward, the bin offsets, out-of-frame flags and sorted
point arrays in the workspace (located by gmi_workspace_layout) against a
numpy counting sort of the same float32 bin keys.  The order of points
inside a bin is not unique (atomic ranks), so the sorted arrays are checked
as a permutation of the input that is consistent with the offsets.  The
plan's nearest-distance bounds are checked by their defining property
against a k-d tree."""
import ctypes

import numpy as np
import pytest
from scipy.spatial import cKDTree

import workloads as wl

pytestmark = pytest.mark.gpu


def bin_keys(points, H, W, b, nbx, nby):
    """Bin of every point as the kernels form it: clamp(floor(x * (1/b)), 0, nb - 1)
    in float32 (1/b is exact for the power-of-two edges), row-major."""
    inv = np.float32(1.0) / np.float32(b)
    x, y = points[:, 0].astype(np.float32), points[:, 1].astype(np.float32)
    fx = np.floor(x * inv)
    fy = np.floor(y * inv)
    fx = np.nan_to_num(np.clip(fx, 0, nbx - 1))
    fy = np.nan_to_num(np.clip(fy, 0, nby - 1))
    return fy.astype(np.int64) * nbx + fx.astype(np.int64)


def run_and_read(im, dev, bin_px=0):
    import torch
    from paper_2012_13257_b300 import _lib
    L = _lib.load()
    p = _lib.make_params(im.sigma, bin_px=bin_px)
    lay = _lib.WsLayout()
    assert L.gmi_workspace_layout(im.N, im.C, im.H, im.W, ctypes.byref(p), ctypes.byref(lay)) == 0
    ws = torch.zeros(lay.total, dtype=torch.uint8, device=dev)
    P = torch.as_tensor(np.ascontiguousarray(im.points), device=dev)
    V = torch.as_tensor(np.ascontiguousarray(im.values), device=dev)
    out = torch.empty((im.H, im.W, im.C), dtype=torch.float32, device=dev)
    p.flags = _lib.FLAG_SYNC_CHECK
    assert L.gmi_forward(P.data_ptr(), V.data_ptr(), im.N, im.C, im.H, im.W, ctypes.byref(p), out.data_ptr(),
                         None, None, ws.data_ptr(), ws.numel(), None) == 0
    torch.cuda.synchronize()
    raw = ws.cpu().numpy()
    nb = lay.nbx * lay.nby

    def view(offset, dtype, count):
        return raw[offset:offset + count * np.dtype(dtype).itemsize].view(dtype)

    run_and_read.ubound = view(lay.ubound, np.float32, lay.wtx * lay.wty * 32)
    run_and_read.sat = view(lay.sat, np.uint32, (lay.nbx + 1) * (lay.nby + 1))
    return (lay, view(lay.off, np.uint32, nb + 1), view(lay.oob, np.uint8, nb),
            view(lay.sxy, np.float32, 2 * im.N).reshape(im.N, 2), view(lay.sval, np.float32, 4 * im.N).reshape(im.N, 4),
            view(lay.perm, np.uint32, im.N))


CASES = [  # (name, image)
    ("ragged_out_of_frame", lambda: wl.tiny_random(2, 500, 37, 53, C=3, sigma=0.7, margin=3.0)),
    ("clustered_c4", lambda: wl.tiny_random(12, 3000, 131, 67, C=4, sigma=1.1, margin=1.0, clustered=True)),
    ("one_row", lambda: wl.tiny_random(7, 50, 1, 100, C=3, sigma=1.0)),
    ("upsample_1024", wl.upsample_1024),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("bin_px", [0, 4])
def test_binning_is_an_exact_counting_sort(cuda_device, name, make, bin_px):
    im = make()
    lay, off, oob, sxy, sval, perm = run_and_read(im, cuda_device, bin_px)
    nb = lay.nbx * lay.nby
    pts = np.ascontiguousarray(im.points, np.float32)
    vals = np.ascontiguousarray(im.values, np.float32)
    keys = bin_keys(pts, im.H, im.W, lay.bin_px, lay.nbx, lay.nby)
    # counts and the exclusive scan, bit for bit
    want_off = np.concatenate([[0], np.cumsum(np.bincount(keys, minlength=nb))]).astype(np.uint32)
    np.testing.assert_array_equal(off, want_off)
    # out-of-frame flags per bin
    outside = ~((pts[:, 0] >= 0) & (pts[:, 0] < im.W) & (pts[:, 1] >= 0) & (pts[:, 1] < im.H))
    want_oob = np.zeros(nb, np.uint8)
    want_oob[keys[outside]] = 1
    np.testing.assert_array_equal(oob, want_oob)
    # the scatter: a permutation of the input, every point inside its bin's range
    assert np.array_equal(np.sort(perm.astype(np.int64)), np.arange(im.N))
    np.testing.assert_array_equal(sxy, pts[perm])
    np.testing.assert_array_equal(sval[:, :im.C], vals[perm])
    assert not sval[:, im.C:].any()   # padding channels are zero
    bin_of_slot = np.repeat(np.arange(nb), np.diff(want_off.astype(np.int64)))
    np.testing.assert_array_equal(keys[perm], bin_of_slot)


BOUND_CASES = [  # (name, image, every point inside the frame)
    ("ragged_out_of_frame", lambda: wl.tiny_random(2, 500, 37, 53, C=3, sigma=0.7, margin=3.0), False),
    ("clustered_far_field", lambda: wl.tiny_random(11, 800, 64, 96, C=3, sigma=2.0, clustered=True), True),
    ("sparse_small_sigma", lambda: wl.tiny_random(10, 800, 64, 96, C=3, sigma=0.5, clustered=True), True),
    ("upsample_1024", wl.upsample_1024, True),
]


@pytest.mark.parametrize("name,make,inside", BOUND_CASES, ids=[c[0] for c in BOUND_CASES])
def test_plan_bounds_cover_the_nearest_distance(cuda_device, name, make, inside):
    """Every near micro-tile's U is at least the squared distance from each of
    its pixels to the nearest point (float64 k-d tree) and at most the
    near-field limit 100 / kappa; +inf marks the far-field micro-tiles.  With
    every point inside the frame (every non-empty bin usable), the ring
    search stops within about sqrt(m)/b + 2 rings, so U <= 2 (t + sqrt(m) +
    3 b)^2 (t the micro-tile's side, m its largest nearest squared distance).
    The search walks at most RINGS bin rings, so a micro-tile may go to the
    far field only when no point lies within RINGS rings of its bins, or when
    that bound exceeds the limit."""
    RINGS = 3
    im = make()
    lay, off = run_and_read(im, cuda_device)[:2]
    U = run_and_read.ubound.astype(np.float64).reshape(lay.wty, lay.wtx, 4, 8)   # [wty, wtx, ly, lx]
    U = U.transpose(0, 2, 1, 3).reshape(lay.wty * 4, lay.wtx * 8)                 # micro-tile rows x columns
    yy, xx = np.meshgrid(np.arange(im.H) + 0.5, np.arange(im.W) + 0.5, indexing="ij")
    d, _ = cKDTree(np.asarray(im.points, np.float64)).query(np.stack([xx.ravel(), yy.ravel()], 1), workers=-1)
    m = (d * d).reshape(im.H, im.W)
    mty, mtx = -(-im.H // lay.mth), -(-im.W // lay.mtw)
    pad = np.full((mty * lay.mth, mtx * lay.mtw), -np.inf)
    pad[:im.H, :im.W] = m
    mmax = pad.reshape(mty, lay.mth, mtx, lay.mtw).max(axis=(1, 3))   # largest m_q per micro-tile
    Ut = U[:mty, :mtx]
    limit = 100.0 / (np.log2(np.e) / (2.0 * im.sigma ** 2))
    near = np.isfinite(Ut)
    assert near.any()
    assert (Ut[near] >= mmax[near] * (1 - 1e-6) - 1e-5).all()
    assert (Ut[near] <= limit * (1 + 1e-6)).all()
    if inside:
        loose = 2.0 * (max(lay.mth, lay.mtw) + np.sqrt(mmax) + 3.0 * lay.bin_px) ** 2
        assert (Ut[near] <= loose[near]).all()
        # points within RINGS bin rings of each micro-tile's own bins (from the
        # bin counts' 2D prefix sum)
        b = lay.bin_px
        counts = np.diff(off.astype(np.int64)).reshape(lay.nby, lay.nbx)
        cs = np.zeros((lay.nby + 1, lay.nbx + 1), np.int64)
        cs[1:, 1:] = counts.cumsum(0).cumsum(1)
        x0 = np.arange(mtx) * lay.mtw
        y0 = np.arange(mty) * lay.mth
        bx0 = np.floor((x0 + 0.5) / b).astype(np.int64)
        bx1 = np.floor((np.minimum(x0 + lay.mtw, im.W) - 0.5) / b).astype(np.int64)
        by0 = np.floor((y0 + 0.5) / b).astype(np.int64)
        by1 = np.floor((np.minimum(y0 + lay.mth, im.H) - 0.5) / b).astype(np.int64)
        xa, xb = np.clip(bx0 - RINGS, 0, lay.nbx), np.clip(bx1 + RINGS + 1, 0, lay.nbx)
        ya, yb = np.clip(by0 - RINGS, 0, lay.nby), np.clip(by1 + RINGS + 1, 0, lay.nby)
        within = (cs[yb][:, xb] - cs[ya][:, xb] - cs[yb][:, xa] + cs[ya][:, xa]) > 0
        assert ((~within[~near]) | (loose[~near] > limit)).all()


def test_summed_area_table_is_exact(cuda_device):
    """With far-field micro-tiles queued (points squeezed into a corner), the
    summed-area table the near kernel's idle warps build equals numpy's 2D
    cumulative sum of the bin counts, entry for entry."""
    rng = np.random.default_rng(71)
    n, H, W = 3000, 150, 190
    pts = rng.uniform(0, 12, (n, 2)).astype(np.float32)
    im = wl.Image(pts, rng.uniform(0, 1, (n, 3)).astype(np.float32), 0.6, H, W)
    lay, off = run_and_read(im, cuda_device)[:2]
    U = run_and_read.ubound
    assert np.isinf(U).any()   # the far field is in use, so the table was built
    counts = np.diff(off.astype(np.int64)).reshape(lay.nby, lay.nbx)
    want = np.zeros((lay.nby + 1, lay.nbx + 1), np.int64)
    want[1:, 1:] = counts.cumsum(0).cumsum(1)
    np.testing.assert_array_equal(run_and_read.sat.reshape(lay.nby + 1, lay.nbx + 1).astype(np.int64), want)
