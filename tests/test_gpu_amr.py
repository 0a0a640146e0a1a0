"""Parity of the adaptive-grid GPU path with the adaptive-grid oracle
(oracle/fc_oracle_amr.c): quadtree (2D) and octree (3D) grids refined
towards the obstacle boundaries with 2:1 balance, hanging nodes as
constraints, Algorithm 1's hierarchy (Sec. 3), fc_options.amr_uniform >= 0.
The octree cases have patches of up to 841 DoFs, factorised in the global
workspace of the patch-rows kernel.

Bounds as for the uniform grids: operator, load and transfers 1e-12; patch
DoF lists identical and owned rows 1e-11; one sweep and a V-cycle 1e-10
relative; coarse solve 1e-11; FGMRES and standalone GMG with the oracle's
iteration counts and the solution within 1e-6."""
import dataclasses

import numpy as np
import pytest
import scipy.sparse.linalg as spl

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
    "ch64": dataclasses.replace(inputs.channel_2d(0, n=64, nlevels=4), amr_uniform=1),
    "ch128": dataclasses.replace(inputs.channel_2d(3, n=128, nlevels=5), amr_uniform=2),
    "ell64": dataclasses.replace(inputs.batch_2d(7), n=(64, 64), nlevels=4, amr_uniform=1),
    "replay": dataclasses.replace(inputs.channel_replay_2d(0, nx=256, ny=64, nlevels=5), amr_uniform=1),
    "oct16": dataclasses.replace(inputs.channel_3d(0, n=16, nlevels=3), amr_uniform=0),
    "oct16p": dataclasses.replace(inputs.porous_3d(1, n=16, nspheres=3, nlevels=3), amr_uniform=1),
    "oct32": dataclasses.replace(inputs.channel_3d(2, n=32, nlevels=4), amr_uniform=1),
}


@pytest.fixture(scope="module")
def oracles():
    return {name: O.AMRMG(p) for name, p in PROBS.items()}


def solver(fc, p):
    return fc.Solver(p)


@pytest.mark.parametrize("name", list(PROBS))
def test_amr_operator_and_load(fc, oracles, name):
    p = PROBS[name]
    s = solver(fc, p)
    mg = oracles[name]
    for lv in range(1, p.nlevels + 1):
        L = mg.levels[lv - 1]
        A, b, _ = L.csr()
        assert s.ndof(lv) == L.ndof
        x = inputs.uniform_array(L.ndof, 17 + lv)
        assert rel(s.apply(x, level=lv).cpu().numpy(), A @ x) <= OPER_TOL, lv
    _, b, _ = mg.fine.csr()
    assert rel(s.rhs().cpu().numpy(), b) <= OPER_TOL


@pytest.mark.parametrize("name", ["ch64", "ell64", "replay", "oct16", "oct16p", "oct32"])
def test_amr_patch_rows(fc, oracles, name):
    p = PROBS[name]
    s = solver(fc, p)
    for lv in (p.nlevels, p.nlevels - 1):
        L = oracles[name].levels[lv - 1]
        rng = np.random.default_rng(lv)
        for node in rng.choice(L.nnodes, min(25, L.nnodes), replace=False):
            rows, dofs, own = L.patch_inverse_rows(int(node))
            d = s.patch_dofs(int(node), level=lv)
            assert np.array_equal(d, dofs), (lv, node)
            g = s.patch_rows(int(node), level=lv)
            assert g.shape == (p.dim + 1, len(dofs))
            for k in range(p.dim + 1):
                if own[k] < 0:
                    assert np.abs(g[k]).max() == 0
                else:
                    assert rel(g[k], rows[k]) <= 1e-11, (lv, node, k, rel(g[k], rows[k]))


@pytest.mark.parametrize("name", list(PROBS))
def test_amr_sweep(fc, oracles, name):
    p = PROBS[name]
    s = solver(fc, p)
    mg = oracles[name]
    for lv in (p.nlevels, 2):
        L = mg.levels[lv - 1]
        x0 = inputs.uniform_array(L.ndof, 31 + lv)
        b = inputs.uniform_array(L.ndof, 41 + lv)
        want = L.sweep(b, x0)
        got = s.smooth(x0, b, level=lv).cpu().numpy()
        assert rel(got - x0, want - x0) <= SWEEP_TOL, lv


@pytest.mark.parametrize("lanes", ["4", "8", "16"])
@pytest.mark.parametrize("name", ["ch128", "oct32"])
def test_amr_sweep_every_lane_count(fc, oracles, name, lanes, monkeypatch):
    """The apply's lanes per patch (chosen by level size) forced to each
    value: the same sweep as the oracle's."""
    monkeypatch.setenv("FC_AMR_LANES", lanes)
    p = PROBS[name]
    s = solver(fc, p)
    L = oracles[name].levels[-1]
    x0 = inputs.uniform_array(L.ndof, 81)
    b = inputs.uniform_array(L.ndof, 82)
    want = L.sweep(b, x0)
    got = s.smooth(x0, b).cpu().numpy()
    assert rel(got - x0, want - x0) <= SWEEP_TOL


@pytest.mark.parametrize("name", ["ch64", "replay", "oct16", "oct32"])
def test_amr_transfers_and_coarse_solve(fc, oracles, name):
    p = PROBS[name]
    s = solver(fc, p)
    mg = oracles[name]
    F, Cc = mg.levels[-1], mg.levels[-2]
    r = inputs.uniform_array(F.ndof, 51)
    assert rel(s.restrict(r).cpu().numpy(), O.restrict(F, Cc, r)) <= OPER_TOL
    e = inputs.uniform_array(Cc.ndof, 52)
    x = inputs.uniform_array(F.ndof, 53)
    assert rel(s.prolong_add(e, x).cpu().numpy(), O.prolong_add(F, Cc, e, x)) <= OPER_TOL
    C1 = mg.levels[0]
    A, _, _ = C1.csr()
    b1 = inputs.uniform_array(C1.ndof, 61)
    assert rel(s.coarse_solve(b1).cpu().numpy(), spl.spsolve(A.tocsc(), b1)) <= 1e-11


@pytest.mark.parametrize("name", list(PROBS))
def test_amr_vcycle_and_fgmres(fc, oracles, name):
    p = PROBS[name]
    s = solver(fc, p)
    mg = oracles[name]
    n = mg.fine.ndof
    b = inputs.uniform_array(n, 71)
    x0 = inputs.uniform_array(n, 72)
    want = mg.vcycle(x0, b)
    assert rel(s.vcycle(x0, b).cpu().numpy() - x0, want - x0) <= SWEEP_TOL
    x_or, its_or, _, _ = mg.fgmres(mg.rhs(), rtol=1e-8)
    x, its, rr = s.solve(s.rhs(), rtol=1e-8)
    assert its == its_or and rr <= 1e-8
    assert rel(x.cpu().numpy(), x_or) <= 1e-6


def test_amr_standalone_gmg(fc):
    """The paper's standalone setting (Sec. 4: V(6,6), damping 0.8, a 1e9
    residual reduction, alpha = 1e-10) on an adaptive channel stand-in: the
    GPU needs the oracle's cycle count."""
    p = dataclasses.replace(inputs.channel_replay_2d(0, nx=256, ny=64, nlevels=5), amr_uniform=1)
    mg = O.AMRMG(p)
    b = mg.rhs()
    x_or, its_or, _ = mg.gmg_solve(b, reduction=1e-9, maxit=80)
    s = solver(fc, p)
    x, its, red = s.gmg_solve(s.rhs(), reduction=1e-9, maxit=80)
    assert its == its_or and red <= 1e-9
    assert rel(x.cpu().numpy(), x_or) <= 1e-6


def test_amr_standalone_gmg_octree(fc):
    """Standalone V(6,6) GMG (damping 0.8, a 1e9 residual reduction) on an
    octree: the 3D duct with one sphere on a 32^3 lattice; the GPU needs the
    oracle's cycle count."""
    p = dataclasses.replace(inputs.channel_3d(2, n=32, nlevels=4, alpha=1e-10), amr_uniform=1,
                            nu_pre=6, nu_post=6)
    mg = O.AMRMG(p)
    b = mg.rhs()
    x_or, its_or, _ = mg.gmg_solve(b, reduction=1e-9, maxit=80)
    s = solver(fc, p)
    x, its, red = s.gmg_solve(s.rhs(), reduction=1e-9, maxit=80)
    assert its == its_or and red <= 1e-9
    assert rel(x.cpu().numpy(), x_or) <= 1e-6


def test_amr_rejects_unsupported(fc):
    p = PROBS["ch64"]
    for kw in ({"prec": "df64"}, {"cache": "matrix"}, {"element": "q2"}, {"galerkin": True}):
        with pytest.raises(fc.FcError):
            fc.Solver(p, **kw)
    with pytest.raises(fc.FcError):
        fc.Solver(dataclasses.replace(inputs.porous_3d(0, n=8, nspheres=2, nlevels=2), amr_uniform=0), prec="fp32")
    s = solver(fc, p)
    assert s.smooth_noalloc_(s.zeros(), s.rhs()) == fc.FC_ERR_INVALID
