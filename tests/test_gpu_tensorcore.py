"""Tensor-core apply of the shared class blocks (fc_options.tc) inside the
float32 correction-form V-cycle, checked against the oracle.

Patches of one class (bit-identical L_i) share one block of owned rows, so
their local solves (Sec. 3.1.2, cache_inverse) form one dense product, which
the library runs as m16n8 MMA tiles: TF32 (rows and residual rounded to
TF32, 2^-11 relative), TF32 split in two terms (float32-class), or BF16
(2^-8 relative).  Cut patches keep the CUDA cores.  Stated errors of one
V-cycle against the oracle's FP64 V-cycle, relative to its correction:
  tf32x3  2e-5   (the float32-row bound; the split products carry ~2^-22)
  tf32    2e-2   (rows and residual each rounded to 2^-11)
  bf16    5e-2   (rows and residual each rounded to 2^-8)
and inside the FP64 FGMRES every mode reaches relative residual 1e-8 with
velocity and pressure within 1e-6 of the oracle (the mixed-precision bar).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_11636_gb300 import inputs
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu

TC_BOUND = {"tf32x3": 2e-5, "tf32": 2e-2, "bf16": 5e-2}


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
    "por3d16": inputs.porous_3d(0, n=16, nspheres=8, nlevels=3),
}


@pytest.fixture(scope="module")
def oracles():
    return {name: O.MG(p) for name, p in PROBS.items()}


@pytest.mark.parametrize("tc", ["tf32x3", "tf32", "bf16"])
@pytest.mark.parametrize("name", list(PROBS))
def test_tc_vcycle_error(fc, oracles, name, tc):
    p = PROBS[name]
    s = fc.Solver(p, prec="fp32", dedup=1, tc=tc)
    mg = oracles[name]
    b = inputs.random_vector(p, 71)
    x0 = inputs.random_vector(p, 72)
    want = mg.vcycle(x0, b)
    got = s.vcycle(x0, b).cpu().numpy()
    err = rel(got - x0, want - x0)
    assert err <= TC_BOUND[tc], (tc, err)
    s.close()


@pytest.mark.parametrize("name", list(PROBS))
def test_tc_split_matches_cuda_cores(fc, name):
    """The two-term TF32 split lands within float32 rounding of the CUDA-core
    float32 apply (same rows, same V-cycle, different summation)."""
    p = PROBS[name]
    s0 = fc.Solver(p, prec="fp32", dedup=1, tc="none")
    s3 = fc.Solver(p, prec="fp32", dedup=1, tc="tf32x3")
    b = inputs.random_vector(p, 81)
    x0 = inputs.random_vector(p, 82)
    v0 = s0.vcycle(x0, b).cpu().numpy()
    v3 = s3.vcycle(x0, b).cpu().numpy()
    assert rel(v3 - x0, v0 - x0) <= 1e-5
    s0.close()
    s3.close()


@pytest.mark.parametrize("tc", ["tf32x3", "tf32", "bf16"])
@pytest.mark.parametrize("name", list(PROBS))
def test_tc_solve(fc, oracles, name, tc):
    p = PROBS[name]
    mg = oracles[name]
    x_ref, _, _, _ = mg.fgmres(mg.rhs(), rtol=1e-10)
    s = fc.Solver(p, prec="fp32", dedup=1, tc=tc)
    x, its, rr = s.solve(s.rhs(), rtol=1e-8, maxit=300)
    assert rr <= 1e-8
    xg = x.cpu().numpy()
    nd = p.dim + 1
    for comp in (list(range(p.dim)), [p.dim]):
        idx = np.concatenate([np.arange(c, len(xg), nd) for c in comp])
        assert rel(xg[idx], x_ref[idx]) <= 1e-6
    s.close()


def test_tc_rejects_bad_mode(fc):
    with pytest.raises(KeyError):
        fc.Solver(PROBS["ch2d"], prec="fp32", tc="fp8")
