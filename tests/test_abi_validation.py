"""Argument checks of the C-ABI, without a GPU.

fc_setup validates the grid, the level set, alpha, the depth and every
option before its first CUDA call, so each rejected argument returns
FC_ERR_INVALID with a message and a handle that fc_destroy releases.  Entry
points given no handle return FC_ERR_INVALID.  fc_footprint_estimate is pure
host arithmetic.
"""
import ctypes as C
import math

import pytest

from paper_2403_11636_gb300 import build, fc


@pytest.fixture(scope="module")
def lib():
    build.build()
    return fc.load()


def valid(dim=3):
    g = fc.FcGrid()
    g.dim = dim
    for k in range(3):
        g.n[k] = 16 if k < dim else 1
        g.lo[k] = 0.0
        g.hi[k] = 1.0
    o = fc.FcOptions()
    fc.load().fc_options_default(C.byref(o))
    shapes = (fc.FcShape * 1)()
    shapes[0].type = 0
    shapes[0].c[0] = shapes[0].c[1] = shapes[0].c[2] = 0.5
    shapes[0].r[0] = 0.2
    ls = fc.FcLevelset(1, C.cast(shapes, C.POINTER(fc.FcShape)))
    return g, ls, shapes, o


def setup_status(lib, g, ls, o, alpha=1e-8, depth=3):
    h = C.c_void_p()
    st = lib.fc_setup(C.byref(h), C.byref(g), C.byref(ls) if ls is not None else None, alpha, depth,
                      C.byref(o), None)
    msg = lib.fc_last_error(h).decode() if h.value else ""
    if h.value:
        assert lib.fc_destroy(h) == fc.FC_OK
    return st, msg


CASES = [
    ("dim 4", lambda g, ls, sh, o: setattr(g, "dim", 4), {}, "dim must be 2 or 3"),
    ("depth 0", lambda g, ls, sh, o: None, {"depth": 0}, "depth out of range"),
    ("depth 64", lambda g, ls, sh, o: None, {"depth": 64}, "depth out of range"),
    ("n not divisible", lambda g, ls, sh, o: g.n.__setitem__(1, 12), {"depth": 4}, "multiple of 2^(depth-1)"),
    ("n zero", lambda g, ls, sh, o: g.n.__setitem__(0, 0), {}, "multiple of 2^(depth-1)"),
    ("empty box", lambda g, ls, sh, o: g.hi.__setitem__(2, 0.0), {}, "empty box"),
    ("alpha 0", lambda g, ls, sh, o: None, {"alpha": 0.0}, "invalid options"),
    ("alpha nan", lambda g, ls, sh, o: None, {"alpha": math.nan}, "invalid options"),
    ("eta 0", lambda g, ls, sh, o: setattr(o, "eta", 0.0), {}, "invalid options"),
    ("omega 0", lambda g, ls, sh, o: setattr(o, "omega", 0.0), {}, "invalid options"),
    ("nu_pre -1", lambda g, ls, sh, o: setattr(o, "nu_pre", -1), {}, "invalid options"),
    ("quad depth 7", lambda g, ls, sh, o: setattr(o, "quad_depth", 7), {}, "invalid options"),
    ("restart 0", lambda g, ls, sh, o: setattr(o, "fgmres_restart", 0), {}, "invalid options"),
    ("restart 257", lambda g, ls, sh, o: setattr(o, "fgmres_restart", 257), {}, "invalid options"),
    ("preset 3", lambda g, ls, sh, o: setattr(o, "bc_preset", 3), {}, "invalid options"),
    ("force kind 4", lambda g, ls, sh, o: setattr(o, "force_kind", 4), {}, "invalid options"),
    ("beta -1", lambda g, ls, sh, o: setattr(o, "nitsche_beta", -1.0), {}, "invalid options"),
    ("dedup 2", lambda g, ls, sh, o: setattr(o, "dedup", 2), {}, "invalid options"),
    ("tc 4", lambda g, ls, sh, o: setattr(o, "tc", 4), {}, "invalid options"),
    ("tc -1", lambda g, ls, sh, o: setattr(o, "tc", -1), {}, "invalid options"),
    ("badcut_frac -1", lambda g, ls, sh, o: setattr(o, "badcut_frac", -1.0), {}, "invalid options"),
    ("badcut_frac 1", lambda g, ls, sh, o: setattr(o, "badcut_frac", 1.0), {}, "invalid options"),
    ("galerkin 2", lambda g, ls, sh, o: setattr(o, "galerkin", 2), {}, "invalid coarse-operator choice"),
    ("galerkin with Q2-Q1", lambda g, ls, sh, o: (setattr(o, "galerkin", 1), setattr(o, "element", 1)), {},
     "need the Q1-Q1 pair"),
    ("cache 3", lambda g, ls, sh, o: setattr(o, "cache", 3), {}, "invalid cache policy or precision"),
    ("prec 9", lambda g, ls, sh, o: setattr(o, "prec", 9), {}, "invalid cache policy or precision"),
    ("fp32 rows with cache_matrix",
     lambda g, ls, sh, o: (setattr(o, "prec", fc.PREC["fp32"]), setattr(o, "cache", fc.CACHE["matrix"])), {},
     "cache_inverse only"),
    ("grid too large", lambda g, ls, sh, o: (g.n.__setitem__(0, 2048), g.n.__setitem__(1, 2048),
                                             g.n.__setitem__(2, 256)), {}, "grid too large"),
    ("negative shape count", lambda g, ls, sh, o: setattr(ls, "nshapes", -1), {}, "bad level set"),
    ("shapes missing", lambda g, ls, sh, o: setattr(ls, "shapes", C.POINTER(fc.FcShape)()), {}, "bad level set"),
    ("ellipse in 3D", lambda g, ls, sh, o: (setattr(sh[0], "type", 1), sh[0].r.__setitem__(1, 0.1)), {},
     "unsupported shape type"),
    ("shape type 2", lambda g, ls, sh, o: setattr(sh[0], "type", 2), {}, "unsupported shape type"),
    ("zero radius", lambda g, ls, sh, o: sh[0].r.__setitem__(0, 0.0), {}, "bad radius"),
]


@pytest.mark.parametrize("name,mutate,kw,message", CASES, ids=[c[0] for c in CASES])
def test_setup_rejects(lib, name, mutate, kw, message):
    g, ls, shapes, o = valid()
    mutate(g, ls, shapes, o)
    st, msg = setup_status(lib, g, ls, o, **kw)
    assert st == fc.FC_ERR_INVALID, (name, st, msg)
    assert message in msg, (name, msg)


def test_ellipse_with_zero_minor_axis_rejected_in_2d(lib):
    g, ls, shapes, o = valid(dim=2)
    shapes[0].type = 1
    shapes[0].r[1] = 0.0
    shapes[0].rot[0] = 1.0
    st, msg = setup_status(lib, g, ls, o)
    assert st == fc.FC_ERR_INVALID and "bad radius" in msg


def test_null_arguments(lib):
    g, ls, shapes, o = valid()
    h = C.c_void_p()
    assert lib.fc_setup(None, C.byref(g), C.byref(ls), 1e-8, 3, C.byref(o), None) == fc.FC_ERR_INVALID
    assert lib.fc_setup(C.byref(h), None, C.byref(ls), 1e-8, 3, C.byref(o), None) == fc.FC_ERR_INVALID
    assert lib.fc_setup(C.byref(h), C.byref(g), C.byref(ls), 1e-8, 3, None, None) == fc.FC_ERR_INVALID
    assert lib.fc_options_default(None) == fc.FC_ERR_INVALID


def test_entry_points_without_a_handle(lib):
    """Every handle-taking call returns FC_ERR_INVALID for a null handle."""
    i, d, ll = C.c_int(), C.c_double(), C.c_longlong()
    sz = (C.c_size_t * 8)()
    calls = [
        lambda: lib.fc_rhs(None, None),
        lambda: lib.fc_residual(None, 1, None, None, None),
        lambda: lib.fc_apply(None, 1, None, None),
        lambda: lib.fc_smooth(None, 2, None, None, 1),
        lambda: lib.fc_smooth_noalloc(None, 2, None, None, 1),
        lambda: lib.fc_restrict(None, 2, None, None),
        lambda: lib.fc_prolong_add(None, 2, None, None),
        lambda: lib.fc_coarse_solve(None, None, None),
        lambda: lib.fc_vcycle(None, None, None),
        lambda: lib.fc_solve(None, None, None, 1e-8, 10, C.byref(i), C.byref(d)),
        lambda: lib.fc_solve_host(None, None, None, 1e-8, 10, C.byref(i), C.byref(d)),
        lambda: lib.fc_gmg_solve(None, None, None, 1e-9, 10, C.byref(i), C.byref(d)),
        lambda: lib.fc_info(None, 1, C.byref(ll), C.byref(ll), sz),
        lambda: lib.fc_patch_rows(None, 1, 0, None),
        lambda: lib.fc_profile_enable(None, 1),
        lambda: lib.fc_profile_read(None, 0, C.byref(ll), C.byref(d), C.byref(d)),
        lambda: lib.fc_sync(None),
        lambda: lib.fc_destroy(None),
        lambda: lib.fc_batch_create(None, None, 0, None),
        lambda: lib.fc_batch_smooth(None, None, None, 1),
        lambda: lib.fc_batch_vcycle(None, None, None),
        lambda: lib.fc_batch_solve(None, None, None, 1e-8, 10, None, None),
        lambda: lib.fc_batch_set_tile(None, 4, 256, 4),
        lambda: lib.fc_batch_sync(None),
        lambda: lib.fc_batch_destroy(None),
    ]
    for k, call in enumerate(calls):
        assert call() == fc.FC_ERR_INVALID, k


def test_failed_setup_leaves_a_handle_that_runs_nothing(lib):
    """Without a GPU, fc_setup stops at its first allocation.  The handle it
    leaves holds partial data: every call that would launch work on it
    returns FC_ERR_INVALID, so no kernel can run on missing buffers."""
    g, ls, shapes, o = valid(dim=2)
    h = C.c_void_p()
    st = lib.fc_setup(C.byref(h), C.byref(g), C.byref(ls), 1e-8, 3, C.byref(o), None)
    assert h.value
    try:
        if st == fc.FC_OK:
            pytest.skip("a GPU is present")
        assert st == fc.FC_ERR_CUDA
        buf = (C.c_double * 4)()
        p = C.cast(buf, C.c_void_p)
        i, d, ll = C.c_int(), C.c_double(), C.c_longlong()
        calls = {
            "rhs": lambda: lib.fc_rhs(h, p),
            "residual": lambda: lib.fc_residual(h, 3, p, p, p),
            "apply": lambda: lib.fc_apply(h, 3, p, p),
            "smooth": lambda: lib.fc_smooth(h, 3, p, p, 1),
            "smooth_noalloc": lambda: lib.fc_smooth_noalloc(h, 3, p, p, 1),
            "restrict": lambda: lib.fc_restrict(h, 3, p, p),
            "prolong": lambda: lib.fc_prolong_add(h, 3, p, p),
            "coarse": lambda: lib.fc_coarse_solve(h, p, p),
            "vcycle": lambda: lib.fc_vcycle(h, p, p),
            "solve": lambda: lib.fc_solve(h, p, p, 1e-8, 10, C.byref(i), C.byref(d)),
            "gmg": lambda: lib.fc_gmg_solve(h, p, p, 1e-9, 10, C.byref(i), C.byref(d)),
            "solve_host": lambda: lib.fc_solve_host(h, p, p, 1e-8, 10, C.byref(i), C.byref(d)),
            "info": lambda: lib.fc_info(h, 3, C.byref(ll), None, None),
            "patch_rows": lambda: lib.fc_patch_rows(h, 3, 0, C.cast(buf, C.POINTER(C.c_double))),
        }
        for name, call in calls.items():
            assert call() == fc.FC_ERR_INVALID, name
            assert b"not set up" in lib.fc_last_error(h), name
        b = C.c_void_p()
        hs = (C.c_void_p * 1)(h.value)
        assert lib.fc_batch_create(C.byref(b), hs, 1, None) == fc.FC_ERR_INVALID
        assert b"not set up" in lib.fc_batch_last_error(b)
        assert lib.fc_batch_destroy(b) == fc.FC_OK
    finally:
        assert lib.fc_destroy(h) == fc.FC_OK


def test_batch_rejects_a_handle_given_twice(lib):
    """A batch uses each problem's level vectors as its workspace, so one
    handle may appear once only.  Without a GPU, fc_setup stops at its first
    allocation but leaves a handle with the problem's parameters, which is
    enough for the batch's argument checks."""
    g, ls, shapes, o = valid(dim=2)
    h = C.c_void_p()
    st = lib.fc_setup(C.byref(h), C.byref(g), C.byref(ls), 1e-8, 3, C.byref(o), None)
    assert h.value
    try:
        if st == fc.FC_OK:
            pytest.skip("a GPU is present")
        b = C.c_void_p()
        hs = (C.c_void_p * 3)(h.value, h.value, h.value)
        assert lib.fc_batch_create(C.byref(b), hs, 3, None) == fc.FC_ERR_INVALID
        assert b"appears twice" in lib.fc_batch_last_error(b)
        assert lib.fc_batch_destroy(b) == fc.FC_OK
        b = C.c_void_p()
        assert lib.fc_batch_create(C.byref(b), hs, 0, None) == fc.FC_ERR_INVALID
        assert lib.fc_batch_destroy(b) == fc.FC_OK
    finally:
        assert lib.fc_destroy(h) == fc.FC_OK


def test_footprint_estimate(lib):
    g, ls, shapes, o = valid()
    assert lib.fc_footprint_estimate(None, 3, C.byref(o)) == 0
    assert lib.fc_footprint_estimate(C.byref(g), 0, C.byref(o)) == 0
    g.dim = 5
    assert lib.fc_footprint_estimate(C.byref(g), 3, C.byref(o)) == 0
    g.dim = 3
    f64 = lib.fc_footprint_estimate(C.byref(g), 3, C.byref(o))
    est = {}
    for name in ("fp32", "bf16", "df64"):
        o.prec = fc.PREC[name]
        est[name] = lib.fc_footprint_estimate(C.byref(g), 3, C.byref(o))
    # reduced-precision rows are built in float64 and then converted: the
    # finest level's float64 rows coexist with the converted rows of every
    # level; narrower rows still need less
    finest, coarser = 17 ** 3 * 402 * 4, 9 ** 3 * 402 * 4
    for name, eb in (("fp32", 4), ("bf16", 2), ("df64", 8)):
        assert est[name] >= finest * 8 + (finest + coarser) * eb, name
    assert est["df64"] > est["fp32"] > est["bf16"] > 0
    assert f64 >= (finest + coarser) * 8
    o.prec = fc.PREC["fp64"]
    g.n[0] = g.n[1] = g.n[2] = 32
    assert 6 < lib.fc_footprint_estimate(C.byref(g), 4, C.byref(o)) / f64 < 10
