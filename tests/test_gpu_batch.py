"""Batched problems (fc_batch_*): every problem of an uneven batch against the
FP64 oracle, and each result independent of the rest of the batch.

The batch runs all problems' sweeps, transfers, coarse solves and Krylov
steps in shared launches; per problem it must compute what the single-problem
path computes: the paper's RA sweep (Sec. 3.1), V-cycle (Sec. 3) and the
FGMRES outer iteration, to the same bounds as the single-problem parity
tests (1e-10 per sweep / V-cycle in FP64, the same iteration counts).
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_11636_gb300 import inputs
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu

SWEEP_TOL = 1e-10


@pytest.fixture(scope="module")
def fc():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2403_11636_gb300 import build, fc as fcmod
    build.build()
    return fcmod


def uneven_2d():
    """Grids 16^2 (3 levels) and 32^2 (4 levels), 1-8 ellipses, alpha in
    {1e-6, 1e-8, 1e-10}, plus an 8^2 problem with a single level (the V-cycle
    is the coarse solve alone)."""
    probs = [inputs.batch_2d(s, sizes=(16, 32)) for s in (0, 2, 3, 5, 7)]
    probs.append(dataclasses.replace(inputs.batch_2d(9, sizes=(8,)), nlevels=1))
    return probs


def small_3d():
    return [inputs.porous_3d(0, n=8, nspheres=6, nlevels=2), inputs.porous_3d(3, n=16, nspheres=10, nlevels=3)]


def make_batch(fc, probs, prec="fp64"):
    solvers = [fc.Solver(p, prec=prec) for p in probs]
    return solvers, fc.Batch(solvers)


def test_batch_layout(fc):
    probs = uneven_2d()
    solvers, B = make_batch(fc, probs)
    assert B.offsets[0] == 0
    for p, s in enumerate(solvers):
        assert B.offsets[p + 1] - B.offsets[p] == s.ndof()
    info = B.info()
    assert info["nprob"] == len(probs) and info["ndof"] == B.offsets[-1]
    assert info["levels_max"] == max(p.nlevels for p in probs)
    # patches of the smoothed finest levels (the one-level problem has none)
    assert info["npatch_finest"] == sum(np.prod([k + 1 for k in p.n[:2]]) for p in probs if p.nlevels > 1)
    tpp, thr, cps = B.tile()
    assert tpp in (1, 2, 4, 8, 16, 32) and thr in (128, 256, 512) and thr * cps <= 2048 and thr // tpp <= 256


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_batch_sweep_parity(fc, which):
    """One and three RA sweeps on every finest level: each problem within
    1e-10 of the oracle's sweep."""
    probs = [p for p in (uneven_2d() if which == "2d" else small_3d()) if p.nlevels > 1]
    solvers, B = make_batch(fc, probs)
    x0 = [inputs.random_vector(p, 31 + k) for k, p in enumerate(probs)]
    bb = [inputs.random_vector(p, 131 + k) for k, p in enumerate(probs)]
    X, Bv = B.pack(x0), B.pack(bb)
    B.smooth_(X, Bv, nsweeps=1)
    got = [v.cpu().numpy() for v in B.unpack(X)]
    B.smooth_(X, Bv, nsweeps=2)
    got3 = [v.cpu().numpy() for v in B.unpack(X)]
    for k, p in enumerate(probs):
        L = O.Level.from_problem(p)
        L.assemble()
        x1 = L.sweep(bb[k], x0[k], mode=0)
        assert rel(got[k] - x0[k], x1 - x0[k]) <= SWEEP_TOL, (which, k)
        x3 = L.sweep(bb[k], L.sweep(bb[k], x1, mode=0), mode=0)
        assert rel(got3[k], x3) <= SWEEP_TOL, (which, k)


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_batch_vcycle_parity(fc, which):
    probs = uneven_2d() if which == "2d" else small_3d()
    solvers, B = make_batch(fc, probs)
    x0 = [inputs.random_vector(p, 71 + k) for k, p in enumerate(probs)]
    bb = [inputs.random_vector(p, 171 + k) for k, p in enumerate(probs)]
    X = B.pack(x0)
    B.vcycle_(X, B.pack(bb))
    for k, (p, v) in enumerate(zip(probs, B.unpack(X))):
        want = O.MG(p).vcycle(x0[k], bb[k])
        assert rel(v.cpu().numpy(), want) <= SWEEP_TOL, (which, k)


def test_batch_fgmres_parity(fc):
    """Per problem: the oracle's iteration count, true residual <= 1e-8 and
    the oracle's solution to 1e-6."""
    probs = uneven_2d()
    solvers, B = make_batch(fc, probs)
    X, its, rr = B.solve(B.rhs(), rtol=1e-8)
    for k, (p, v) in enumerate(zip(probs, B.unpack(X))):
        mg = O.MG(p)
        x_or, its_or, _, _ = mg.fgmres(mg.rhs(), rtol=1e-8)
        assert its[k] == its_or, (k, its[k], its_or)
        assert rr[k] <= 1e-8
        assert rel(v.cpu().numpy(), x_or) <= 1e-6


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_batch_mixed_precision_solve(fc, prec):
    """Reduced-precision rows in the batched solve: relative residual 1e-8
    and every problem within 1e-6 of the oracle's FP64 solution."""
    probs = uneven_2d()
    solvers, B = make_batch(fc, probs, prec=prec)
    X, its, rr = B.solve(B.rhs(), rtol=1e-8, maxit=400)
    for k, (p, v) in enumerate(zip(probs, B.unpack(X))):
        assert rr[k] <= 1e-8
        mg = O.MG(p)
        x_or, _, _, _ = mg.fgmres(mg.rhs(), rtol=1e-10)
        assert rel(v.cpu().numpy(), x_or) <= 1e-6, (prec, k)
        # the single-problem path with the same rows needs as many cycles,
        # give or take the rounding order of the float32 sums
        _, its1, _ = solvers[k].solve(solvers[k].rhs(), rtol=1e-8, maxit=400)
        assert abs(its1 - its[k]) <= 1, (prec, k, its1, its[k])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_member_independence(fc, prec):
    """A problem's solve and V-cycle are bit-identical alone and in the batch
    (same tile)."""
    probs = uneven_2d()
    solvers, B = make_batch(fc, probs, prec=prec)
    B.set_tile(8, 256, 4)
    bb = B.rhs()
    X, its, _ = B.solve(bb, rtol=1e-8, maxit=400)
    x0 = [inputs.random_vector(p, 91 + k) for k, p in enumerate(probs)]
    XV = B.pack(x0)
    B.vcycle_(XV, bb)
    for k in (0, 2, len(probs) - 1):
        one = fc.Batch([solvers[k]])
        one.set_tile(8, 256, 4)
        b1 = solvers[k].rhs()
        x1, its1, _ = one.solve(b1, rtol=1e-8, maxit=400)
        assert its1[0] == its[k]
        assert np.array_equal(x1.cpu().numpy(), B.unpack(X)[k].cpu().numpy())
        xv = one.pack([x0[k]])
        one.vcycle_(xv, b1)
        assert np.array_equal(xv.cpu().numpy(), B.unpack(XV)[k].cpu().numpy())
        one.close()


def test_batch_tiles_agree(fc):
    """Every tile candidate computes the same sweep up to rounding order."""
    probs = uneven_2d()[:4]
    solvers, B = make_batch(fc, probs)
    x0 = B.pack([inputs.random_vector(p, 11 + k) for k, p in enumerate(probs)])
    bb = B.pack([inputs.random_vector(p, 21 + k) for k, p in enumerate(probs)])
    ref = None
    for tpp in (1, 2, 4, 8, 16, 32):
        for thr, cps in ((128, 16), (512, 2)):
            if thr // tpp > 256:
                continue
            B.set_tile(tpp, thr, cps)
            X = B.smooth_(x0.clone(), bb, nsweeps=2).cpu().numpy()
            if ref is None:
                ref = X
            assert rel(X, ref) <= 1e-13


def test_batch_invalid(fc):
    s2 = fc.Solver(inputs.batch_2d(0, sizes=(16,)))
    s3 = fc.Solver(inputs.porous_3d(0, n=8, nspheres=6, nlevels=2))
    with pytest.raises(fc.FcError) as e:
        fc.Batch([s2, s3])
    assert e.value.code == fc.FC_ERR_INVALID
    sd = fc.Solver(inputs.batch_2d(0, sizes=(16,)), prec="df64")
    with pytest.raises(fc.FcError) as e:
        fc.Batch([sd])
    assert e.value.code == fc.FC_ERR_INVALID
    sm = fc.Solver(inputs.batch_2d(0, sizes=(16,)), cache="matrix")
    with pytest.raises(fc.FcError):
        fc.Batch([sm])
    B = fc.Batch([s2])
    with pytest.raises(fc.FcError):
        B.set_tile(3, 256, 4)
    with pytest.raises(fc.FcError):
        B.set_tile(1, 512, 4)   # 512 patches per pass
