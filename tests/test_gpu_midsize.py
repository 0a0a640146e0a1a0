"""Parity with the full oracle on a mid-size 3D problem: the benchmark's
40-sphere porous geometry on a 32^3 background grid with 4 levels (35,937
patches on the finest level, 143,748 DoFs).  The oracle assembles every
level and caches every patch inverse, so whole sweeps, V-cycles and FGMRES
solves are compared, for FP64 rows and for the float-pair rows the benchmark
times: per sweep and per V-cycle within 1e-10 relative, FGMRES with the
oracle's iteration count (paper Sec. 3.1 eq. iteration and eq. smoother;
Sec. 4 for the iteration counts), reduced-precision rows within the
mixed-precision bounds (relative residual 1e-8, velocity and pressure within
1e-6 of the oracle)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_11636_gb300 import inputs
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu

SWEEP_TOL = 1e-10


@pytest.fixture(scope="module")
def mid():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2403_11636_gb300 import build, fc
    build.build()
    p = inputs.porous_3d(0, n=32, nlevels=4)
    mg = O.MG(p)                      # every level assembled, inverse rows cached
    b = mg.rhs()
    x_or, its_or, rr_or, _ = mg.fgmres(b, rtol=1e-8)
    return {"p": p, "fc": fc, "mg": mg, "b": b, "x": x_or, "its": its_or, "solvers": {}}


def solver(mid, prec, cache="inverse"):
    key = (prec, cache)
    if key not in mid["solvers"]:
        mid["solvers"][key] = mid["fc"].Solver(mid["p"], prec=prec, cache=cache, dedup=0)
    return mid["solvers"][key]


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("level", [4, 3])
def test_mid_sweep(mid, prec, level):
    """Two sweeps on the finest (32^3) and the next (16^3) level."""
    p, mg = mid["p"], mid["mg"]
    s = solver(mid, prec)
    L = mg.levels[level - 1]
    x0 = inputs.random_vector(p, 40 + level, level=level)
    b = inputs.random_vector(p, 50 + level, level=level)
    want = L.sweep(b, L.sweep(b, x0))
    got = s.smooth(x0, b, level=level, nsweeps=2).cpu().numpy()
    assert rel(got - x0, want - x0) <= SWEEP_TOL


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_mid_vcycle(mid, prec):
    p, mg = mid["p"], mid["mg"]
    s = solver(mid, prec)
    x0 = inputs.random_vector(p, 61)
    b = inputs.random_vector(p, 62)
    want = mg.vcycle(x0, b)
    got = s.vcycle(x0, b).cpu().numpy()
    assert rel(got - x0, want - x0) <= SWEEP_TOL


@pytest.mark.parametrize("prec,cache", [("fp64", "inverse"), ("df64", "inverse"), ("fp64", "matrix")])
def test_mid_fgmres_iterations(mid, prec, cache):
    """Same iteration count as the oracle, true residual <= 1e-8, and the
    oracle's solution to 1e-6."""
    s = solver(mid, prec, cache)
    x, its, rr = s.solve(s.rhs(), rtol=1e-8)
    assert its == mid["its"], (its, mid["its"])
    assert rr <= 1e-8
    assert rel(x.cpu().numpy(), mid["x"]) <= 1e-6


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_mid_mixed_precision(mid, prec):
    """Float32 / bfloat16 rows inside the FP64 FGMRES: relative residual
    1e-8; velocity and pressure each within 1e-6 of the oracle's solution
    (taken to 1e-10 so that its own error does not count)."""
    p, mg = mid["p"], mid["mg"]
    x_ref, _, _, _ = mg.fgmres(mid["b"], rtol=1e-10)
    s = solver(mid, prec)
    x, its, rr = s.solve(s.rhs(), rtol=1e-8, maxit=300)
    assert rr <= 1e-8
    xg = x.cpu().numpy()
    nd = p.dim + 1
    for comp in (list(range(p.dim)), [p.dim]):
        idx = np.concatenate([np.arange(c, len(xg), nd) for c in comp])
        assert rel(xg[idx], x_ref[idx]) <= 1e-6
