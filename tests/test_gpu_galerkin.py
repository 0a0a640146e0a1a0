"""Galerkin coarse operators (fc_options.galerkin = 1) against the oracle's
R L_f P hierarchy (or_galerkin): the coarser grids take the product of the
next finer operator with the V-cycle's transfers instead of their own
rediscretisation (Sec. 3, hierarchy of coarser discretisations).

Bounds as for the rediscretised hierarchy: coarse operators 1e-12 (rounding
order only); sweeps on a coarse level and V-cycles 1e-10; FGMRES with the
oracle's iteration count, relative residual 1e-8 and the solution within
1e-6.  Shared class blocks (coarse cell classes from the children's) change
nothing bit for bit; float32 rows reach the mixed-precision bar."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_11636_gb300 import inputs
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu

OPER_TOL = 1e-12
SWEEP_TOL = 1e-10


@pytest.fixture(scope="module")
def fc():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2403_11636_gb300 import build, fc as fcmod
    build.build()
    return fcmod


PROBS = {
    "ch2d": inputs.channel_2d(0, n=32, nlevels=3),
    "por3d": inputs.porous_3d(0, n=16, nspheres=8, nlevels=3),
}


@pytest.fixture(scope="module")
def oracles():
    return {name: O.MG(p, galerkin=True) for name, p in PROBS.items()}


@pytest.mark.parametrize("name", list(PROBS))
def test_galerkin_coarse_operators(fc, oracles, name):
    p = PROBS[name]
    s = fc.Solver(p, galerkin=True)
    mg = oracles[name]
    for lv in range(1, p.nlevels + 1):
        A, _, _ = mg.levels[lv - 1].csr()
        x = inputs.random_vector(p, 17 + lv, level=lv)
        assert rel(s.apply(x, level=lv).cpu().numpy(), A @ x) <= OPER_TOL, lv


@pytest.mark.parametrize("name", list(PROBS))
def test_galerkin_coarse_sweep_and_vcycle(fc, oracles, name):
    p = PROBS[name]
    s = fc.Solver(p, galerkin=True)
    mg = oracles[name]
    lv = p.nlevels - 1
    x0 = inputs.random_vector(p, 41, level=lv)
    b = inputs.random_vector(p, 42, level=lv)
    got = s.smooth(x0, b, level=lv).cpu().numpy()
    assert rel(got - x0, mg.levels[lv - 1].sweep(b, x0) - x0) <= SWEEP_TOL
    b = inputs.random_vector(p, 71)
    x0 = inputs.random_vector(p, 72)
    want = mg.vcycle(x0, b)
    assert rel(s.vcycle(x0, b).cpu().numpy() - x0, want - x0) <= SWEEP_TOL


@pytest.mark.parametrize("name", list(PROBS))
def test_galerkin_fgmres(fc, oracles, name):
    p = PROBS[name]
    s = fc.Solver(p, galerkin=True)
    mg = oracles[name]
    x_or, its_or, _, _ = mg.fgmres(mg.rhs(), rtol=1e-8)
    x, its, rr = s.solve(s.rhs(), rtol=1e-8)
    assert its == its_or and rr <= 1e-8
    assert rel(x.cpu().numpy(), x_or) <= 1e-6


def test_galerkin_shared_classes_change_nothing(fc):
    p = PROBS["por3d"]
    s0 = fc.Solver(p, galerkin=True, dedup=0)
    s1 = fc.Solver(p, galerkin=True, dedup=1)
    b = inputs.random_vector(p, 81)
    x0 = inputs.random_vector(p, 82)
    np.testing.assert_array_equal(s1.vcycle(x0, b).cpu().numpy(), s0.vcycle(x0, b).cpu().numpy())
    assert s1.info()["bytes"][1] < s0.info()["bytes"][1]


@pytest.mark.parametrize("prec", ["fp32", "df64"])
def test_galerkin_reduced_precision_rows(fc, oracles, prec):
    p = PROBS["por3d"]
    s = fc.Solver(p, galerkin=True, prec=prec)
    mg = oracles["por3d"]
    x_or, _, _, _ = mg.fgmres(mg.rhs(), rtol=1e-10)
    x, its, rr = s.solve(s.rhs(), rtol=1e-8)
    assert rr <= 1e-8
    assert rel(x.cpu().numpy(), x_or) <= 1e-6
