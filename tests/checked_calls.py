"""Runs the library's call paths through the checked build (bounds checks that
record instead of trapping, guard areas after every workspace region) and
checks each call's workspace afterwards; the results are compared with the
FP64 oracle.  Run as a separate process with GMI_CHECKED=1 (the package then
loads libgmi_checked.so); prints one line per path and exits non-zero on the
first failure.  Used by test_checked_gpu.py."""
import ctypes
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
import workloads as wl  # noqa: E402
import paper_2012_13257_b300 as gmi  # noqa: E402
from paper_2012_13257_b300 import _lib  # noqa: E402
from gpu_helpers import TOL_FWD, to_dev  # noqa: E402

DEV = torch.device("cuda", 0)
L = _lib.load()
assert _lib.CHECKED and L.gmi_is_checked_build() == 1, "not the checked build"


def workspace():
    """The package's per-stream workspace the last call used."""
    (buf,) = list(gmi._ws_buffers.values())
    return buf


def check_ws(name, N, C, H, W, sigma, mode, k=6.0, variant=0):
    torch.cuda.synchronize()
    buf = workspace()
    p = _lib.make_params(sigma, k, mode, 0, 0, variant)
    rep = (ctypes.c_uint32 * 4)()
    st = L.gmi_check_workspace(N, C, H, W, ctypes.byref(p), buf.data_ptr(), buf.numel(), None, rep)
    assert st == 0, "%s: gmi_check_workspace status %d, report %s" % (name, st, list(rep))
    assert list(rep) == [0, 0, 0, 0], (name, list(rep))


def fwd_case(name, im, mode="exact", k=6.0, variant=0, graph=False, gather=None):
    gmi.release_workspaces()
    if gather:
        gmi.set_gather(gather)
    P, V = to_dev(im.points, DEV), to_dev(im.values, DEV)
    out = gmi.interpolate(P, V, im.sigma, im.H, im.W, mode=mode, radius_sigmas=k, variant=variant, graph=graph,
                          check=not graph)
    check_ws(name, im.N, im.values.shape[1], im.H, im.W, im.sigma, _lib.MODE_EXACT if mode == "exact" else
             _lib.MODE_TRUNCATED, k, variant)
    ref = oracle.forward(im.points, im.values, im.H, im.W, im.sigma, mode=oracle.EXACT if mode == "exact" else
                         oracle.TRUNCATED, k=k)
    keep = ref["skipped"] < 1e-3
    err = np.abs(out.cpu().numpy().astype(np.float64) - ref["image"])[keep].max()
    assert err <= TOL_FWD, (name, err)
    if gather:
        gmi.set_gather("auto")
    print("ok", name, "max err %.2e" % err, flush=True)


def main():
    # forward: dense, ragged, far field (points in one corner), clustered
    # (split tiles), truncated, both gathers, micro-tile variants, graph replay
    fwd_case("forward dense 64x64", wl.small_uniform())
    fwd_case("forward ragged clustered", wl.tiny_random(3, 900, 61, 77, C=3, sigma=0.7, clustered=True))
    corner = wl.tiny_random(4, 300, 70, 90, C=3, sigma=0.8, clustered=True)
    corner = wl.Image((corner.points * 0.2).astype(np.float32), corner.values, corner.sigma, corner.H, corner.W)
    fwd_case("forward far field", corner)
    fwd_case("forward dense cluster (splits)", wl.tiny_random(5, 6000, 64, 64, C=4, sigma=2.0, clustered=True))
    fwd_case("forward truncated", wl.tiny_random(6, 700, 50, 66, C=2, sigma=0.9), mode="truncated", k=3.0)
    fwd_case("forward direct gather", wl.tiny_random(7, 800, 64, 80, C=3, sigma=1.0), gather="direct")
    for v in (2, 3, 4):
        fwd_case("forward variant %d" % v, wl.tiny_random(8 + v, 600, 45, 61, C=3, sigma=1.2, clustered=True),
                 variant=v)
    fwd_case("forward graph replay", wl.tiny_random(12, 700, 64, 64, C=3, sigma=1.0), graph=True)

    # the guard check itself: a byte changed (from the host) in the guard area
    # after the status words (the workspace's first region, 256 bytes) is
    # reported as guard 1; the next call writes the guards again
    im = wl.small_uniform()
    fwd_case("forward before a changed guard", im)
    buf = workspace()
    buf[256 + 8] ^= 0x5A
    torch.cuda.synchronize()
    p = _lib.make_params(im.sigma, 6.0, _lib.MODE_EXACT, 0, 0, 0)
    rep = (ctypes.c_uint32 * 4)()
    st = L.gmi_check_workspace(im.N, 3, im.H, im.W, ctypes.byref(p), buf.data_ptr(), buf.numel(), None, rep)
    assert st == 10 and (rep[0] & 32) and rep[3] == 1, ("changed guard not reported", st, list(rep))
    fwd_case("forward after a changed guard", im)
    print("ok a changed guard is reported", flush=True)

    # backward (exact, far field included)
    gmi.release_workspaces()
    im, g = wl.fd_subcase()
    P, V = to_dev(im.points, DEV), to_dev(im.values, DEV)
    img, den, shift = gmi.interpolate(P, V, im.sigma, im.H, im.W, return_aux=True)
    gp, gv, gs = gmi.interpolate_backward(P, V, im.sigma, im.H, im.W, img, den, shift, to_dev(g, DEV), check=True)
    check_ws("backward", im.N, 3, im.H, im.W, im.sigma, _lib.MODE_EXACT)
    ref = oracle.backward(im.points, im.values, im.H, im.W, im.sigma, g)
    e = np.abs(gp.cpu().numpy() - ref["points"]).max() / np.abs(ref["points"]).max()
    assert e <= 1e-3, ("backward", e)
    print("ok backward rel err %.2e" % e, flush=True)

    # per-point sigma and full covariance, exact and truncated, forward and backward
    for kind, mode in ((1, "exact"), (3, "exact"), (1, "truncated"), (3, "truncated")):
        gmi.release_workspaces()
        im = wl.tiny_random(20 + kind, 500, 45, 61, C=3, sigma=1.2, clustered=True)
        sig = wl.point_sigmas(30, im.N, 0.4, 1.2) if kind == 1 else wl.point_cov(31, im.N, 0.4, 1.2, rmax=0.9)
        bound = 1.2 if kind == 1 else wl.cov_bound(sig)
        k = 6.0 if mode == "exact" else 3.0
        P, V, S = to_dev(im.points, DEV), to_dev(im.values, DEV), to_dev(sig, DEV)
        img, den = gmi.interpolate_pp(P, V, S, bound, im.H, im.W, radius_sigmas=k, mode=mode, return_aux=True,
                                      check=True)
        gup = to_dev(np.random.default_rng(kind).standard_normal((im.H, im.W, 3)).astype(np.float32), DEV)
        gmi.interpolate_backward_pp(P, V, S, bound, im.H, im.W, img, den, gup, radius_sigmas=k, mode=mode,
                                    check=True)
        md = _lib.MODE_EXACT if mode == "exact" else _lib.MODE_TRUNCATED
        check_ws("per-point kind %d %s" % (kind, mode), im.N, 3, im.H, im.W, bound, md, k)
        fwd = oracle.forward_pp if kind == 1 else oracle.forward_cov
        ref = fwd(im.points, im.values, sig, im.H, im.W, mode=oracle.EXACT if mode == "exact" else oracle.TRUNCATED,
                  k=k)
        keep = ref["skipped"] < 1e-3
        err = np.abs(img.cpu().numpy().astype(np.float64) - ref["image"])[keep].max()
        assert err <= TOL_FWD, ("per-point", kind, mode, err)
        print("ok per-point kind %d %s max err %.2e" % (kind, mode, err), flush=True)

    # batched forward and backward through one plan
    ims = [wl.tiny_random(40 + b, 300 + 200 * b, 40 + 9 * b, 50 + 7 * b, C=3, sigma=0.6 + 0.3 * b, clustered=b % 2 == 1)
           for b in range(5)]
    plan = gmi.BatchPlan(8, 4000, 200 * 200, C=3)
    descs = [{"points": to_dev(m.points, DEV), "values": to_dev(m.values, DEV), "sigma": m.sigma, "H": m.H,
              "W": m.W} for m in ims]
    outs = plan.forward(descs)
    torch.cuda.synchronize()
    rep = (ctypes.c_uint32 * 4)()
    st = L.gmi_batch_check_workspace(plan._h, None, rep)
    assert st == 0 and list(rep) == [0, 0, 0, 0], ("batched", st, list(rep))
    for m, o in zip(ims, outs):
        ref = oracle.forward(m.points, m.values, m.H, m.W, m.sigma)
        assert np.abs(o.cpu().numpy() - ref["image"]).max() <= TOL_FWD
    print("ok batched forward", flush=True)
    print("ALL OK", flush=True)


if __name__ == "__main__":
    main()
