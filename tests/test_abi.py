"""The C-ABI library loads and exports every entry point include/gmi.h
declares; host-side argument checks reject bad calls before any GPU work.
No compute call is made (this runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2012_13257_b300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gmi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*(gmi_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gmi_forward", "gmi_backward", "gmi_workspace_size", "gmi_forward_batched",
                     "gmi_server_create", "gmi_server_submit", "gmi_server_wait"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(declared_functions()) == set(_lib.SIGNATURES)


def test_version_and_status_strings():
    lib = _lib.load()
    assert b"sm_103a" in lib.gmi_version()
    for code, name in _lib.STATUS_NAMES.items():
        assert lib.gmi_status_string(code).decode() == name


def test_params_default():
    p = _lib.Params()
    assert _lib.load().gmi_params_default(ctypes.byref(p)) == 0
    assert p.sigma == 1.0 and p.radius_sigmas == 6.0 and p.mode == 0 and p.flags == 0


def _ws(N, C, H, W, **kw):
    p = _lib.make_params(kw.pop("sigma", 1.0), **kw)
    n = ctypes.c_size_t(0)
    st = _lib.load().gmi_workspace_size(N, C, H, W, ctypes.byref(p), ctypes.byref(n))
    return st, n.value


def test_workspace_size_checks():
    st, n = _ws(4096, 3, 64, 64)
    assert st == 0 and n > 0 and n % 256 == 0
    st2, n2 = _ws(8192, 3, 64, 64)
    assert st2 == 0 and n2 > n
    assert _ws(-1, 3, 8, 8)[0] == 1
    assert _ws(10, 3, 0, 8)[0] == 1
    assert _ws(10, 5, 8, 8)[0] == 7
    assert _ws(10, 0, 8, 8)[0] == 7
    assert _ws(10, 3, 8, 8, sigma=0.0)[0] == 1
    assert _ws(10, 3, 8, 8, sigma=float("nan"))[0] == 1
    assert _ws(10, 3, 8, 8, radius_sigmas=-1.0)[0] == 1
    assert _ws(10, 3, 8, 8, mode=7)[0] == 1
    assert _ws(10, 3, 8, 8, flags=0x4)[0] == 1       # unknown flag bit
    assert _ws(10, 3, 8, 8, flags=_lib.FLAG_GRAPH | _lib.FLAG_SYNC_CHECK)[0] == 0


def test_flag_values_match_the_header():
    src = open(os.path.join(ROOT, "include", "gmi.h")).read()
    defs = dict(re.findall(r"#define\s+GMI_(FLAG_[A-Z_]+)\s+(0x[0-9a-fA-F]+)u", src))
    assert {k: int(v, 16) for k, v in defs.items()} == {"FLAG_SYNC_CHECK": _lib.FLAG_SYNC_CHECK,
                                                       "FLAG_GRAPH": _lib.FLAG_GRAPH}


def test_forward_rejects_bad_arguments_without_launching():
    lib = _lib.load()
    p = _lib.make_params(1.0)
    assert lib.gmi_forward(None, None, 10, 3, 8, 8, ctypes.byref(p), None, None, None, None, 0, None) == 1
    bad = _lib.make_params(-2.0)
    assert lib.gmi_forward(None, None, 10, 3, 8, 8, ctypes.byref(bad), 256, None, None, 256, 1 << 20, None) == 1
    # workspace too small / misaligned: rejected before anything is enqueued (the
    # fake pointers are never dereferenced)
    assert lib.gmi_forward(256, 256, 10, 3, 8, 8, ctypes.byref(p), 256, None, None, 256, 16, None) == 3
    assert lib.gmi_forward(256, 256, 10, 3, 8, 8, ctypes.byref(p), 256, None, None, 257, 1 << 20, None) == 3


def test_package_fails_loudly_without_the_library(monkeypatch):
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", "/nonexistent/libgmi.so")
    with pytest.raises(ImportError):
        _lib.load()


def test_autotune_rejects_bad_arguments_without_launching():
    lib = _lib.load()
    p = _lib.make_params(1.0)
    best = _lib.Params()
    bins = (ctypes.c_int * 2)(0, 2)
    assert lib.gmi_autotune(256, 256, 10, 3, 8, 8, ctypes.byref(p), bins, 0, 3, ctypes.byref(best), None, None) == 1
    assert lib.gmi_autotune(256, 256, 10, 3, 8, 8, ctypes.byref(p), bins, 2, 0, ctypes.byref(best), None, None) == 1
    assert lib.gmi_autotune(256, 256, 10, 3, 8, 8, ctypes.byref(p), bins, 2, 3, None, None, None) == 1
    bad = (ctypes.c_int * 1)(4096)
    assert lib.gmi_autotune(256, 256, 10, 3, 8, 8, ctypes.byref(p), bad, 1, 3, ctypes.byref(best), None, None) == 1


@pytest.mark.parametrize("kind", ["pp", "aniso", "cov"])
def test_per_point_calls_reject_bad_arguments_without_launching(kind):
    """A missing or misaligned sigma array is GMI_ERR_INVALID_ARG, and a
    short workspace GMI_ERR_WORKSPACE, in either mode; all are found on the
    host before anything is enqueued (the fake pointers are never
    dereferenced)."""
    lib = _lib.load()
    fwd, bwd = getattr(lib, "gmi_forward_" + kind), getattr(lib, "gmi_backward_" + kind)
    for mode in (_lib.MODE_EXACT, _lib.MODE_TRUNCATED):
        p = _lib.make_params(1.0, mode=mode)
        assert fwd(256, 256, None, 10, 3, 8, 8, ctypes.byref(p), 256, None, 256, 1 << 20, None) == 1
        assert fwd(256, 256, 258, 10, 3, 8, 8, ctypes.byref(p), 256, None, 256, 1 << 20, None) == 1
        assert bwd(256, 256, None, 10, 3, 8, 8, ctypes.byref(p), 256, 256, 256, None, None, None, 256, 1 << 20,
                   None) == 1
        assert bwd(256, 256, 258, 10, 3, 8, 8, ctypes.byref(p), 256, 256, 256, None, None, None, 256, 1 << 20,
                   None) == 1
        # the workspace is checked too
        assert fwd(256, 256, 256, 10, 3, 8, 8, ctypes.byref(p), 256, None, 256, 16, None) == 3


def test_stacked_calls_reject_bad_arguments_without_launching():
    """No plan, B < 1 or a NULL sigma array: GMI_ERR_INVALID_ARG on the host."""
    lib = _lib.load()
    sig = (ctypes.c_float * 2)(1.0, 1.0)
    assert lib.gmi_forward_stacked(None, 256, 256, 2, 10, 8, 8, sig, 256, None, None, 1, None) == 1
    assert lib.gmi_backward_stacked(None, 256, 256, 2, 10, 8, 8, sig, 256, 256, 256, 256, None, None, None,
                                    None) == 1


def test_workspace_layout_is_consistent_without_a_gpu():
    """gmi_workspace_layout is host arithmetic: its total equals
    gmi_workspace_size, its regions are 256-byte aligned, in order and large
    enough for their arrays, and bad arguments are rejected."""
    from paper_2012_13257_b300 import _lib
    L = _lib.load()
    for N, C, H, W, sigma, bin_px in ((262144, 3, 1024, 1024, 1.0, 0), (500, 4, 37, 53, 0.7, 4), (1, 1, 1, 1, 2.0, 0)):
        p = _lib.make_params(sigma, bin_px=bin_px)
        lay = _lib.WsLayout()
        assert L.gmi_workspace_layout(N, C, H, W, ctypes.byref(p), ctypes.byref(lay)) == 0
        size = ctypes.c_size_t(0)
        assert L.gmi_workspace_size(N, C, H, W, ctypes.byref(p), ctypes.byref(size)) == 0
        assert lay.total == size.value
        nb = lay.nbx * lay.nby
        assert lay.nbx == -(-W // lay.bin_px) and lay.nby == -(-H // lay.bin_px)
        assert lay.wtx == -(-W // (8 * lay.mtw)) and lay.wty == -(-H // (4 * lay.mth))
        regions = [(lay.off, 4 * (nb + 1)), (lay.oob, nb), (lay.sxy, 8 * N), (lay.sval, 16 * N), (lay.perm, 4 * N),
                   (lay.ubound, 4 * 32 * lay.wtx * lay.wty)]
        for start, nbytes in regions:
            assert start % 256 == 0 and start + nbytes <= lay.total
        assert lay.off < lay.oob and lay.sxy < lay.sval < lay.perm
    p = _lib.make_params(1.0)
    lay = _lib.WsLayout()
    assert L.gmi_workspace_layout(10, 0, 8, 8, ctypes.byref(p), ctypes.byref(lay)) != 0   # C = 0
    assert L.gmi_workspace_layout(10, 3, 8, 8, ctypes.byref(p), None) == 1                  # no output
    bad = _lib.make_params(-1.0)
    assert L.gmi_workspace_layout(10, 3, 8, 8, ctypes.byref(bad), ctypes.byref(lay)) == 1   # sigma <= 0


def test_checked_build_exports_and_layout():
    """The checked build (libgmi_checked.so) exports the same entry points,
    says it is checked, and sizes its workspaces larger (a guard area after
    every region); the normal build answers the check calls with
    GMI_ERR_UNSUPPORTED before touching anything."""
    path = os.path.join(ROOT, "paper_2012_13257_b300", "libgmi_checked.so")
    if not os.path.exists(path):
        from paper_2012_13257_b300 import build as b
        b.build(checked=True)
    chk = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(chk, n)]
    assert not missing, missing
    lib = _lib.load()
    assert chk.gmi_is_checked_build() == 1 and lib.gmi_is_checked_build() == 0
    p = _lib.make_params(1.0)
    for fn in (lib.gmi_workspace_size, chk.gmi_workspace_size):
        fn.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_lib.Params),
                       ctypes.POINTER(ctypes.c_size_t)]
    a, b = ctypes.c_size_t(0), ctypes.c_size_t(0)
    assert lib.gmi_workspace_size(1000, 3, 64, 64, ctypes.byref(p), ctypes.byref(a)) == 0
    assert chk.gmi_workspace_size(1000, 3, 64, 64, ctypes.byref(p), ctypes.byref(b)) == 0
    assert b.value >= a.value + 17 * 256
    rep = (ctypes.c_uint32 * 4)()
    assert lib.gmi_check_workspace(1000, 3, 64, 64, ctypes.byref(p), 256, a.value, None, rep) == 7
    assert lib.gmi_batch_check_workspace(256, None, rep) == 7


def test_wait_limit_setting_is_host_only():
    """gmi_set_wait_polls only records the limit for later launches: it needs
    no GPU, takes any value (negative restores the defaults) and always
    returns GMI_OK."""
    lib = _lib.load()
    for polls in (0, 1, 10_000, 1 << 40, -1):
        assert lib.gmi_set_wait_polls(polls) == 0
    assert lib.gmi_set_wait_polls(-1) == 0
