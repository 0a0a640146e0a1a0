"""The banded LDL^T factorisation of the 3D patch blocks against the pivoted
dense LU it falls back to, and against the oracle.

In 3D every patch's owned rows (all row precisions) and every cache_matrix
record come from a banded LDL^T of the equilibrated velocity block; a patch
whose block meets a pivot <= FC_LDL_MIN_PIVOT (1e-14) is built by the dense
pivoted LU instead, through a redo list (owned rows) or a side array of
dense records with a node list (cache_matrix).  The porous problems of the
test sizes have positive definite blocks throughout (checked with the
oracle's own matrices), so these tests set FC_LDL_MIN_PIVOT above 1, which
sends every patch down the fallback, and compare the two paths patch by
patch and sweep by sweep, each also against the oracle.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_11636_gb300 import inputs
from tests.gpu_util import oracle_rows_in_slots, rel

pytestmark = pytest.mark.gpu

ROW_TOL = 1e-11
SWEEP_TOL = 1e-10


@pytest.fixture(scope="module")
def fc():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2403_11636_gb300 import build, fc as fcmod
    build.build()
    return fcmod


def problem():
    return inputs.porous_3d(0, n=16, nspheres=8, nlevels=3)


def solver_all_dense(fc, p, **kw):
    """A solver built with every patch sent to the dense pivoted LU."""
    old = os.environ.get("FC_LDL_MIN_PIVOT")
    os.environ["FC_LDL_MIN_PIVOT"] = "2.0"
    try:
        return fc.Solver(p, **kw)
    finally:
        if old is None:
            del os.environ["FC_LDL_MIN_PIVOT"]
        else:
            os.environ["FC_LDL_MIN_PIVOT"] = old


def nn_of(p):
    """Patches (pressure nodes) of the finest level."""
    return int(np.prod([k + 1 for k in p.level_n(p.nlevels)]))


def test_band_and_dense_rows_agree_on_every_patch(fc):
    p = problem()
    band = fc.Solver(p, prec="fp64", dedup=0)
    dense = solver_all_dense(fc, p, prec="fp64", dedup=0)
    assert band.info()["bytes"][5] == 0
    assert dense.info()["bytes"][5] >= nn_of(p)  # every stored patch took the dense LU
    nn = nn_of(p)
    worst = 0.0
    for node in range(nn):
        a, b = band.patch_rows(node), dense.patch_rows(node)
        for k in range(p.dim + 1):
            if np.abs(b[k]).max() == 0:
                assert np.abs(a[k]).max() == 0, (node, k)
            else:
                worst = max(worst, rel(a[k], b[k]))
    assert worst <= ROW_TOL, worst
    # both against the oracle on sampled patches (cut and uncut)
    L = O.Level.from_problem(p)
    L.assemble()
    rng = np.random.default_rng(3)
    for node in rng.choice(nn, 12, replace=False):
        o = oracle_rows_in_slots(L, p, p.level_n(p.nlevels), int(node))
        for s in (band, dense):
            g = s.patch_rows(int(node))
            for k in range(p.dim + 1):
                if np.abs(o[k]).max() > 0:
                    assert rel(g[k], o[k]) <= ROW_TOL, (int(node), k)
    band.close()
    dense.close()


def test_cache_matrix_band_and_dense_records_agree(fc):
    """cache_matrix: the banded records and the dense records (all patches
    through the dense node list) give the same sweep, and both the oracle's."""
    p = problem()
    band = fc.Solver(p, cache="matrix", dedup=0)
    dense = solver_all_dense(fc, p, cache="matrix", dedup=0)
    assert band.info()["bytes"][5] == 0
    assert dense.info()["bytes"][5] >= nn_of(p)
    L = O.Level.from_problem(p)
    L.assemble()
    x0 = inputs.random_vector(p, 41)
    b = inputs.random_vector(p, 42)
    x_or = L.sweep(b, x0, mode=0)
    xb = band.smooth(x0, b, nsweeps=1).cpu().numpy()
    xd = dense.smooth(x0, b, nsweeps=1).cpu().numpy()
    assert rel(xb - x0, x_or - x0) <= SWEEP_TOL
    assert rel(xd - x0, x_or - x0) <= SWEEP_TOL
    assert rel(xb - x0, xd - x0) <= SWEEP_TOL
    # a V-cycle through every level's records
    xbv = band.vcycle(x0, b).cpu().numpy()
    xdv = dense.vcycle(x0, b).cpu().numpy()
    assert rel(xbv - x0, xdv - x0) <= SWEEP_TOL
    band.close()
    dense.close()


def test_shared_class_records_with_dense_fallback(fc):
    """With shared class blocks (dedup) the node -> record map goes through
    the patch classes; forcing the dense records must not change a sweep."""
    p = problem()
    band = fc.Solver(p, cache="matrix", dedup=1)
    dense = solver_all_dense(fc, p, cache="matrix", dedup=1)
    x0 = inputs.random_vector(p, 43)
    b = inputs.random_vector(p, 44)
    xb = band.smooth(x0, b, nsweeps=2).cpu().numpy()
    xd = dense.smooth(x0, b, nsweeps=2).cpu().numpy()
    assert rel(xb - x0, xd - x0) <= SWEEP_TOL
    band.close()
    dense.close()


def test_cache_none_band_and_dense_agree(fc):
    """cache_none: the banded on-the-fly solve, and the dense one for every
    patch (all listed at setup), give the oracle's sweep."""
    p = problem()
    band = fc.Solver(p, cache="none")
    dense = solver_all_dense(fc, p, cache="none")
    assert band.info()["bytes"][5] == 0
    assert dense.info()["bytes"][5] >= nn_of(p)
    L = O.Level.from_problem(p)
    L.assemble()
    x0 = inputs.random_vector(p, 45)
    b = inputs.random_vector(p, 46)
    x_or = L.sweep(b, x0, mode=0)
    xb = band.smooth(x0, b, nsweeps=1).cpu().numpy()
    xd = dense.smooth(x0, b, nsweeps=1).cpu().numpy()
    assert rel(xb - x0, x_or - x0) <= SWEEP_TOL
    assert rel(xd - x0, x_or - x0) <= SWEEP_TOL
    band.close()
    dense.close()
