"""Parity of the CUDA path (through the C-ABI) with the FP64 CPU oracle.

Every comparison uses the same seeded inputs on both sides.  FP64 paths must
agree to 1e-10 relative per smoother sweep and reach the same FGMRES
iteration counts; operator applications, transfers and the coarse solve are
held to tighter bounds that only rounding order can explain.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_11636_gb300 import inputs
from tests.gpu_util import oracle_patch_update, oracle_rows_in_slots, rel

pytestmark = pytest.mark.gpu

SWEEP_TOL = 1e-10      # per-sweep FP64 parity
OPER_TOL = 1e-12       # operator / transfer parity (rounding order only)


@pytest.fixture(scope="module")
def fc():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2403_11636_gb300 import build, fc as fcmod
    build.build()
    return fcmod


def problems():
    return {
        "ch2d": inputs.channel_2d(0, n=32, nlevels=3),
        "ch2d_s3": inputs.channel_2d(3, n=16, nlevels=2, alpha=1e-10),
        "por3d": inputs.porous_3d(0, n=8, nspheres=6, nlevels=2),
        "ch3d": dataclass_replace(inputs.porous_3d(5, n=8, nspheres=3, nlevels=2), preset=0),
        "ell2d": inputs.batch_2d(7),
    }


def dataclass_replace(p, **kw):
    import dataclasses
    return dataclasses.replace(p, **kw)


PROBS = problems()


@pytest.mark.parametrize("name", list(PROBS))
def test_rhs_and_operator(fc, name):
    p = PROBS[name]
    s = fc.Solver(p)
    L = O.Level.from_problem(p)
    A, b_or, fixed = L.csr()
    b_gpu = s.rhs().cpu().numpy()
    assert rel(b_gpu, b_or) <= OPER_TOL * 10
    x = inputs.random_vector(p, 17)
    y_gpu = s.apply(x).cpu().numpy()
    assert rel(y_gpu, A @ x) <= OPER_TOL
    r_gpu = s.residual(x, b_or).cpu().numpy()
    assert rel(r_gpu, b_or - A @ x) <= OPER_TOL


@pytest.mark.parametrize("name", list(PROBS))
def test_coarse_levels_operator(fc, name):
    p = PROBS[name]
    s = fc.Solver(p)
    for lv in range(1, p.nlevels):
        L = O.Level.from_problem(p, lv)
        A, _, _ = L.csr()
        x = inputs.random_vector(p, 23, level=lv)
        assert rel(s.apply(x, level=lv).cpu().numpy(), A @ x) <= OPER_TOL


@pytest.mark.parametrize("name", ["ch2d", "por3d", "ell2d"])
@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
def test_patch_rows(fc, name, prec):
    """Cached owned rows of L_i^{-1} (cache_inverse) equal the oracle's: the
    FP64 build and the float-pair build (df64 rows; fp32 rows are the pair
    rows rounded to float32)."""
    tol = {"fp64": 1e-11, "df64": 1e-11, "fp32": 2e-7}[prec]
    p = PROBS[name]
    s = fc.Solver(p, prec=prec)
    L = O.Level.from_problem(p)
    L.assemble()
    rng = np.random.default_rng(0)
    nn = np.prod([k + 1 for k in p.level_n(p.nlevels)])
    for node in rng.choice(nn, 24, replace=False):
        g = s.patch_rows(int(node))
        o = oracle_rows_in_slots(L, p, p.level_n(p.nlevels), int(node))
        for k in range(p.dim + 1):
            if np.abs(o[k]).max() == 0:
                assert np.abs(g[k]).max() == 0
            else:
                assert rel(g[k], o[k]) <= tol, (prec, node, k, rel(g[k], o[k]))


@pytest.mark.parametrize("cache", ["inverse", "matrix", "none"])
@pytest.mark.parametrize("name", list(PROBS))
def test_sweep_parity(fc, name, cache):
    """One RA sweep on the finest level: relative 2-norm difference <= 1e-10."""
    p = PROBS[name]
    s = fc.Solver(p, cache=cache)
    L = O.Level.from_problem(p)
    L.assemble()
    x0 = inputs.random_vector(p, 31)
    b = inputs.random_vector(p, 32)
    x_or = L.sweep(b, x0, mode=0)
    x_gpu = s.smooth(x0, b, nsweeps=1).cpu().numpy()
    assert rel(x_gpu - x0, x_or - x0) <= SWEEP_TOL
    # three sweeps in a row
    x_or3 = L.sweep(b, L.sweep(b, x_or, mode=0), mode=0)
    x_gpu3 = s.smooth(x0, b, nsweeps=3).cpu().numpy()
    assert rel(x_gpu3, x_or3) <= SWEEP_TOL


COARSER = {"ch2d": PROBS["ch2d"], "por3d16": inputs.porous_3d(0, n=16, nspheres=8, nlevels=3)}


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("name", list(COARSER))
def test_sweep_parity_coarser_level(fc, name, prec):
    """A sweep on the level below the finest (a smoothed level that the
    V-cycle reaches through the restriction)."""
    p = COARSER[name]
    s = fc.Solver(p, prec=prec)
    lv = p.nlevels - 1
    assert lv >= 2
    L = O.Level.from_problem(p, lv)
    L.assemble()
    x0 = inputs.random_vector(p, 41, level=lv)
    b = inputs.random_vector(p, 42, level=lv)
    got = s.smooth(x0, b, level=lv).cpu().numpy()
    assert rel(got - x0, L.sweep(b, x0) - x0) <= SWEEP_TOL


@pytest.mark.parametrize("name", ["ch2d", "por3d"])
def test_transfers(fc, name):
    p = PROBS[name]
    s = fc.Solver(p)
    F = O.Level.from_problem(p, p.nlevels)
    Cc = O.Level.from_problem(p, p.nlevels - 1)
    r = inputs.random_vector(p, 51)
    assert rel(s.restrict(r).cpu().numpy(), O.restrict(F, Cc, r)) <= OPER_TOL
    e = inputs.random_vector(p, 52, level=p.nlevels - 1)
    x = inputs.random_vector(p, 53)
    assert rel(s.prolong_add(e, x).cpu().numpy(), O.prolong_add(F, Cc, e, x)) <= OPER_TOL


@pytest.mark.parametrize("name", ["ch2d", "por3d", "ell2d"])
def test_coarse_solve(fc, name):
    p = PROBS[name]
    s = fc.Solver(p)
    C1 = O.Level.from_problem(p, 1)
    A, _, _ = C1.csr()
    b = inputs.random_vector(p, 61, level=1)
    x_gpu = s.coarse_solve(b).cpu().numpy()
    x_or = O.dense_solve(A.toarray(), b)
    assert rel(x_gpu, x_or) <= 1e-11


@pytest.mark.parametrize("cache,prec", [("inverse", "fp64"), ("inverse", "df64"), ("matrix", "fp64"),
                                        ("none", "fp64")])
@pytest.mark.parametrize("name", ["ch2d", "por3d", "ell2d"])
def test_vcycle_parity(fc, name, cache, prec):
    """One V-cycle against the oracle's: FP64 rows with every cache policy,
    and the float-pair rows the benchmark times (pair smoothing phases,
    FP64 transfers and coarse solve)."""
    p = PROBS[name]
    s = fc.Solver(p, cache=cache, prec=prec)
    mg = O.MG(p)
    b = inputs.random_vector(p, 71)
    x0 = inputs.random_vector(p, 72)
    got = s.vcycle(x0, b).cpu().numpy()
    want = mg.vcycle(x0, b)
    assert rel(got, want) <= SWEEP_TOL
    assert rel(got - x0, want - x0) <= SWEEP_TOL


@pytest.mark.parametrize("cache,prec", [("inverse", "fp64"), ("inverse", "df64"), ("matrix", "fp64")])
@pytest.mark.parametrize("name", ["ch2d", "por3d", "ch3d", "ell2d"])
def test_fgmres_parity(fc, name, cache, prec):
    """Same iteration count as the oracle, true residual <= 1e-8, and the same
    solution to the accuracy the tolerance allows."""
    p = PROBS[name]
    s = fc.Solver(p, cache=cache, prec=prec)
    mg = O.MG(p)
    b = mg.rhs()
    x_or, its_or, rel_or, _ = mg.fgmres(b, rtol=1e-8)
    x_gpu, its_gpu, rel_gpu = s.solve(s.rhs(), rtol=1e-8)
    assert its_gpu == its_or
    assert rel_gpu <= 1e-8
    assert rel(x_gpu.cpu().numpy(), x_or) <= 1e-6


@pytest.mark.parametrize("prec", ["df64"])
@pytest.mark.parametrize("name", ["ch2d", "por3d"])
def test_df64_sweep_parity(fc, name, prec):
    """Rows stored and applied as float32 pairs (about 48-bit significand)
    keep the per-sweep FP64 parity bound."""
    p = PROBS[name]
    s = fc.Solver(p, prec=prec)
    L = O.Level.from_problem(p)
    L.assemble()
    x0 = inputs.random_vector(p, 81)
    b = inputs.random_vector(p, 82)
    x_or = L.sweep(b, x0)
    assert rel(s.smooth(x0, b).cpu().numpy() - x0, x_or - x0) <= SWEEP_TOL


@pytest.mark.parametrize("prec", ["fp32", "bf16", "df64"])
@pytest.mark.parametrize("name", ["ch2d", "por3d"])
def test_mixed_precision_solve(fc, name, prec):
    """Reduced-precision patch rows inside the FP64 FGMRES: relative residual
    1e-8 and velocity / pressure within 1e-6 of the oracle's solution."""
    p = PROBS[name]
    s = fc.Solver(p, prec=prec)
    mg = O.MG(p)
    b = mg.rhs()
    x_or, _, _, _ = mg.fgmres(b, rtol=1e-10)
    x_gpu, its, rr = s.solve(s.rhs(), rtol=1e-8, maxit=300)
    assert rr <= 1e-8
    xg = x_gpu.cpu().numpy()
    nd = p.dim + 1
    for comp in (list(range(p.dim)), [p.dim]):
        idx = np.concatenate([np.arange(c, len(xg), nd) for c in comp])
        assert rel(xg[idx], x_or[idx]) <= 1e-6


def test_order_independence_bitwise(fc):
    """The sweep result does not depend on launch order: two runs are bit
    identical (no atomics on the owned DoFs)."""
    p = PROBS["por3d"]
    s = fc.Solver(p)
    x0 = inputs.random_vector(p, 91)
    b = inputs.random_vector(p, 92)
    a1 = s.smooth(x0, b).cpu().numpy()
    a2 = s.smooth(x0, b).cpu().numpy()
    np.testing.assert_array_equal(a1, a2)


def test_invalid_arguments_rejected(fc):
    """Host-side validation returns FC_ERR_INVALID without touching the GPU."""
    import dataclasses
    p = dataclasses.replace(inputs.channel_2d(0, n=30, nlevels=3))
    with pytest.raises(fc.FcError) as e:
        fc.Solver(p)
    assert e.value.code == fc.FC_ERR_INVALID
    p2 = dataclasses.replace(inputs.channel_2d(0, n=16, nlevels=2), alpha=-1.0)
    with pytest.raises(fc.FcError):
        fc.Solver(p2)
    with pytest.raises(fc.FcError):
        fc.Solver(inputs.porous_3d(0, n=8, nspheres=2, nlevels=2), cache="matrix", prec="fp32")


def test_binding_rejects_bad_vectors(fc):
    """Vectors of the wrong length, type, layout or memory are rejected by
    the binding before a pointer reaches the library; valid calls still run."""
    import torch
    p = inputs.channel_2d(0, n=16, nlevels=2)
    s = fc.Solver(p)
    n = s.ndof()
    good = s.zeros()
    bad = {
        "short": torch.zeros(n - 1, dtype=torch.float64, device="cuda"),
        "host": torch.zeros(n, dtype=torch.float64),
        "float32": torch.zeros(n, dtype=torch.float32, device="cuda"),
        "strided": torch.zeros(2 * n, dtype=torch.float64, device="cuda")[::2],
    }
    for name, v in bad.items():
        with pytest.raises(fc.FcError) as e:
            s.smooth_(v, good)
        assert e.value.code == fc.FC_ERR_INVALID, name
        with pytest.raises(fc.FcError):
            s.smooth_noalloc_(good, v)
    with pytest.raises(fc.FcError):
        s.residual(bad["short"], good)
    with pytest.raises(fc.FcError):
        s.restrict(good, level=1)
    with pytest.raises(fc.FcError):
        s.solve_host(np.zeros(n - 1), np.zeros(n))
    b = s.rhs()
    x = s.smooth(good, b)
    assert x.shape == (n,) and torch.isfinite(x).all()
    _, its, rr = s.solve(b, rtol=1e-8)
    assert rr <= 1e-8
    B = fc.Batch([s])
    with pytest.raises(fc.FcError):
        B.smooth_(bad["host"], good)
    with pytest.raises(fc.FcError):
        B.pack([bad["short"]])
    B.close()
    s.close()


def test_no_obstacle_and_one_level(fc):
    """Degenerate cases: no obstacle at all; a one-level hierarchy (direct
    solve only, FGMRES converges in one step)."""
    import dataclasses
    p = dataclasses.replace(inputs.channel_2d(0, n=16, nlevels=2), shapes=np.zeros((0, 9)))
    s = fc.Solver(p)
    mg = O.MG(p)
    x_or, its_or, _, _ = mg.fgmres(mg.rhs(), rtol=1e-8)
    x, its, rr = s.solve(s.rhs(), rtol=1e-8)
    assert its == its_or and rr <= 1e-8
    p1 = dataclasses.replace(inputs.channel_2d(0, n=8, nlevels=1))
    s1 = fc.Solver(p1)
    x, its, rr = s1.solve(s1.rhs(), rtol=1e-10)
    assert its == 1 and rr <= 1e-10


def test_ragged_and_anisotropic_grid(fc):
    """Non-square grid (n_x != n_y, h_x != h_y) and an ellipse crossing cells."""
    import dataclasses
    p = dataclasses.replace(inputs.batch_2d(3), n=(48, 16), hi=(2.2, 0.41), nlevels=2,
                            shapes=np.array([[1.0, 0.5, 0.2, 0.0, 0.08, 0.05, 0.0, 0.8, 0.6]]))
    s = fc.Solver(p)
    L = O.Level.from_problem(p)
    A, b, _ = L.csr()
    x0 = inputs.random_vector(p, 101)
    assert rel(s.apply(x0).cpu().numpy(), A @ x0) <= OPER_TOL
    assert rel(s.smooth(x0, b).cpu().numpy() - x0, L.sweep(b, x0) - x0) <= SWEEP_TOL


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("name", ["ch2d", "por3d", "ell2d"])
def test_shared_class_blocks_change_nothing(fc, name, prec):
    """Patches with bit-identical blocks L_i share one stored block (dedup=1);
    the results are bit-identical to one block per patch (dedup=0), and far
    fewer blocks are factored."""
    p = PROBS[name]
    s1 = fc.Solver(p, prec=prec, dedup=1)
    s0 = fc.Solver(p, prec=prec, dedup=0)
    x0 = inputs.random_vector(p, 111)
    b = inputs.random_vector(p, 112)
    np.testing.assert_array_equal(s1.smooth(x0, b, nsweeps=2).cpu().numpy(),
                                  s0.smooth(x0, b, nsweeps=2).cpu().numpy())
    nn = np.prod([k + 1 for k in p.level_n(p.nlevels)])
    for node in np.random.default_rng(3).choice(nn, 16, replace=False):
        np.testing.assert_array_equal(s1.patch_rows(int(node)), s0.patch_rows(int(node)))
    assert s1.info()["bytes"][1] <= s0.info()["bytes"][1]


@pytest.mark.parametrize("nx,ny,nlev", [(128, 32, 3), (256, 64, 4), (512, 128, 6)])
def test_standalone_gmg_replay(fc, nx, ny, nlev):
    """Standalone GMG in the paper's setting (Sec. 4: V(6,6), damping 0.8, a
    1e9 residual reduction, alpha = 1e-10) on the channel stand-in: the GPU
    needs the same number of cycles as the oracle."""
    p = inputs.channel_replay_2d(0, nx=nx, ny=ny, nlevels=nlev)
    mg = O.MG(p)
    b = mg.rhs()
    x_or, its_or, red_or = mg.gmg_solve(b, reduction=1e-9, maxit=60)
    s = fc.Solver(p)
    x_gpu, its, red = s.gmg_solve(s.rhs(), reduction=1e-9, maxit=60)
    assert red <= 1e-9 and its == its_or
    assert rel(x_gpu.cpu().numpy(), x_or) <= 1e-6


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("name", ["ch2d", "por3d", "ell2d"])
def test_float32_vcycle_error(fc, name, prec):
    """Reduced-precision rows: the V-cycle runs in the float32 correction
    form (float32 residuals, transfers and patch solves on the correction,
    float64 anchor b - L x0 and float64 accumulation of x).  Stated error
    against the oracle's FP64 V-cycle on the same input: the correction
    within 2e-5 (float32 rows) / 2e-2 (bfloat16 rows) relative."""
    p = PROBS[name]
    s = fc.Solver(p, prec=prec)
    mg = O.MG(p)
    b = inputs.random_vector(p, 71)
    x0 = inputs.random_vector(p, 72)
    want = mg.vcycle(x0, b)
    got = s.vcycle(x0, b).cpu().numpy()
    err = rel(got - x0, want - x0)
    assert err <= (2e-5 if prec == "fp32" else 2e-2), err


def test_float32_build_falls_back_on_ill_conditioned_patches(fc):
    """Float32 / bfloat16 rows come from a float32 factorisation with
    iterative refinement; where the refinement cannot converge (an
    equilibrated block too ill-conditioned for float32 factors, here a badly
    cut patch of an alpha = 1e-10 geometry) the patch is rebuilt by the
    float-pair elimination.  Every stored row then matches the float-pair
    build of the same problem to float32 rounding."""
    p = inputs.batch_2d(63)
    s32 = fc.Solver(p, prec="fp32")
    sdf = fc.Solver(p, prec="df64")
    assert s32.info()["bytes"][5] >= 1          # at least one patch fell back
    nn = (p.n[0] + 1) * (p.n[1] + 1)
    for node in [1583, 1518, 1519, 1648, 7, nn // 2]:
        a, b = s32.patch_rows(node), sdf.patch_rows(node)
        den = np.abs(b).max()
        assert den == 0 or np.abs(a - b).max() <= 2e-7 * den, node
    # same iteration count as the float-pair rows
    _, i32, r32 = s32.solve(s32.rhs(), rtol=1e-8, maxit=400)
    _, idf, _ = sdf.solve(sdf.rhs(), rtol=1e-8, maxit=400)
    assert r32 <= 1e-8 and abs(i32 - idf) <= 1
