"""Parity of the Q2-Q1 (Taylor-Hood) GPU path with the Q2-Q1 oracle.

The element pair with Q2 velocities and Q1 pressures, patches of the Q2
nodes 2a-4 .. 2a+4 and the pressures a-1 .. a+1 around each vertex a, each
Q2 node written by the vertex at the lower corner of its cell, edge or face
(fc_options.element = 1), in 2D (9 owned rows over 171 slots) and 3D (25
owned rows over 2214 slots, the velocity block factored by a banded LU).
Same bounds as the Q1-Q1 parity tests: operator, transfers 1e-12; sweeps
and V-cycles 1e-10 relative; FGMRES and standalone GMG with the oracle's
iteration counts.  Patch rows: 1e-11, or 2e-15 x the condition number of
the equilibrated patch block where that is larger (Q2-Q1 blocks have a zero
pressure block and cond up to ~5e7 on cut patches)."""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_11636_gb300 import inputs
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu

SWEEP_TOL = 1e-10
OPER_TOL = 1e-12


@pytest.fixture(scope="module")
def fc():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2403_11636_gb300 import build, fc as fcmod
    build.build()
    return fcmod


PROBS = {
    "ch2d": inputs.channel_2d(0, n=16, nlevels=3),
    "ell2d": dataclasses.replace(inputs.batch_2d(7), n=(32, 32), nlevels=3),
    "ragged": dataclasses.replace(inputs.batch_2d(3), n=(48, 16), hi=(2.2, 0.41), nlevels=2,
                                  shapes=np.array([[1.0, 0.5, 0.2, 0.0, 0.08, 0.05, 0.0, 0.8, 0.6]])),
    "por3d4": inputs.porous_3d(0, n=4, nspheres=2, nlevels=2),
    "por3d8": inputs.porous_3d(0, n=8, nspheres=4, nlevels=3),
    "duct3d": dataclasses.replace(inputs.porous_3d(2, n=8, nspheres=3, nlevels=2), n=(8, 4, 4),
                                  hi=(2.0, 1.0, 1.0), preset=0),
}
ROWS_CASES = ["ch2d", "ell2d", "por3d4", "por3d8", "duct3d"]


@pytest.fixture(scope="module")
def oracles():
    return {name: O.Q2MG(p) for name, p in PROBS.items()}


def solver(fc, p):
    return fc.Solver(p, element="q2")


@pytest.mark.parametrize("name", list(PROBS))
def test_q2_rhs_and_operator(fc, oracles, name):
    p = PROBS[name]
    s = solver(fc, p)
    mg = oracles[name]
    for lv in range(1, p.nlevels + 1):
        L = mg.levels[lv - 1]
        A, b, _ = L.csr()
        assert s.ndof(lv) == L.ndof
        x = inputs.uniform_array(L.ndof, 17 + lv)
        assert rel(s.apply(x, level=lv).cpu().numpy(), A @ x) <= OPER_TOL
    A, b, _ = mg.fine.csr()
    assert rel(s.rhs().cpu().numpy(), b) <= 10 * OPER_TOL


def expected_rows(L, vert):
    """The oracle's owned rows of the patch of vertex `vert` in the library's
    slot order: velocity (Q2 node of the 9^d box, x fastest, component inner),
    then the 3^d pressures; rows of constrained owned DoFs are zero."""
    dim = L.dim
    nf = [2 * k + 1 for k in L.n]
    nv1 = [k + 1 for k in L.n]
    a = [vert % nv1[0], (vert // nv1[0]) % nv1[1], vert // (nv1[0] * nv1[1]) if dim == 3 else 0]
    nsv = 9 ** dim * dim
    ns, nr = nsv + 3 ** dim, (1 << dim) * dim + 1
    rows, dofs, own = L.patch_inverse_rows(int(vert))
    pos = {int(d): q for q, d in enumerate(dofs)}
    want = np.zeros((nr, ns))
    for slot in range(ns):
        if slot < nsv:
            pn, c = divmod(slot, dim)
            off = (pn % 9, (pn // 9) % 9, pn // 81)
            idx = [2 * a[k] - 4 + off[k] for k in range(dim)]
            if any(not 0 <= idx[k] < nf[k] for k in range(dim)):
                continue
            node = idx[0] + nf[0] * (idx[1] + (nf[1] * idx[2] if dim == 3 else 0))
            d = node * dim + c
        else:
            t = slot - nsv
            off = (t % 3, (t // 3) % 3, t // 9)
            idx = [a[k] - 1 + off[k] for k in range(dim)]
            if any(not 0 <= idx[k] < nv1[k] for k in range(dim)):
                continue
            d = L.nv + idx[0] + nv1[0] * (idx[1] + (nv1[1] * idx[2] if dim == 3 else 0))
        q = pos.get(d)
        if q is None:
            continue
        for k in range(nr):
            if own[k] >= 0:
                want[k, slot] = rows[k, q]
    return want


def rows_tolerance(L, vert):
    """Rows of two exact LU solves differ by about cond x machine epsilon.
    Equilibrated Q2-Q1 patch blocks (zero pressure block) reach cond ~ 5e7 on
    cut patches at alpha = 1e-8 (the Q1-Q1 blocks stay near 40), so the
    bound is max(1e-11, 2e-15 x cond_1(D L_i D)), D = (row max |L_i|)^-1/2."""
    Li, _, _ = L.patch_matrix(int(vert))
    d = 1.0 / np.sqrt(np.abs(Li).max(axis=1))
    return max(1e-11, 2e-15 * np.linalg.cond(d[:, None] * Li * d[None, :], 1))


@pytest.mark.parametrize("name", ROWS_CASES)
def test_q2_patch_rows(fc, oracles, name):
    p = PROBS[name]
    s = solver(fc, p)
    L = oracles[name].fine
    rng = np.random.default_rng(0)
    for vert in rng.choice(L.np, min(20 if p.dim == 2 else 10, L.np), replace=False):
        g = s.patch_rows(int(vert))
        want = expected_rows(L, int(vert))
        assert g.shape == want.shape
        tol = rows_tolerance(L, vert)
        for k in range(want.shape[0]):
            if np.abs(want[k]).max() == 0:
                assert np.abs(g[k]).max() == 0, (vert, k)
            else:
                assert rel(g[k], want[k]) <= tol, (vert, k, rel(g[k], want[k]), tol)


@pytest.mark.parametrize("name", list(PROBS))
def test_q2_sweep_parity(fc, oracles, name):
    p = PROBS[name]
    s = solver(fc, p)
    L = oracles[name].fine
    x0 = inputs.uniform_array(L.ndof, 31)
    b = inputs.uniform_array(L.ndof, 32)
    want = L.sweep(b, x0)
    got = s.smooth(x0, b, nsweeps=1).cpu().numpy()
    assert rel(got - x0, want - x0) <= SWEEP_TOL
    want3 = L.sweep(b, L.sweep(b, want))
    got3 = s.smooth(x0, b, nsweeps=3).cpu().numpy()
    assert rel(got3, want3) <= SWEEP_TOL


@pytest.mark.parametrize("name", ["ch2d", "por3d4"])
def test_q2_sweep_order_independent_bitwise(fc, name):
    p = PROBS[name]
    s = solver(fc, p)
    n = s.ndof()
    x0 = inputs.uniform_array(n, 91)
    b = inputs.uniform_array(n, 92)
    a1 = s.smooth(x0, b).cpu().numpy()
    a2 = s.smooth(x0, b).cpu().numpy()
    np.testing.assert_array_equal(a1, a2)


@pytest.mark.parametrize("name", ["ch2d", "ell2d", "por3d8", "duct3d"])
def test_q2_transfers_and_coarse_solve(fc, oracles, name):
    p = PROBS[name]
    s = solver(fc, p)
    mg = oracles[name]
    F, C = mg.levels[-1], mg.levels[-2]
    r = inputs.uniform_array(F.ndof, 51)
    assert rel(s.restrict(r).cpu().numpy(), O.q2_restrict(F, C, r)) <= OPER_TOL
    e = inputs.uniform_array(C.ndof, 52)
    x = inputs.uniform_array(F.ndof, 53)
    assert rel(s.prolong_add(e, x).cpu().numpy(), O.q2_prolong_add(F, C, e, x)) <= OPER_TOL
    C1 = mg.levels[0]
    A, _, _ = C1.csr()
    b1 = inputs.uniform_array(C1.ndof, 61)
    import scipy.sparse.linalg as spl
    assert rel(s.coarse_solve(b1).cpu().numpy(), spl.spsolve(A.tocsc(), b1)) <= 1e-11


@pytest.mark.parametrize("name", ["ch2d", "ell2d", "por3d8", "duct3d"])
def test_q2_vcycle_parity(fc, oracles, name):
    p = PROBS[name]
    s = solver(fc, p)
    mg = oracles[name]
    n = mg.fine.ndof
    b = inputs.uniform_array(n, 71)
    x0 = inputs.uniform_array(n, 72)
    want = mg.vcycle(x0, b)
    got = s.vcycle(x0, b).cpu().numpy()
    assert rel(got - x0, want - x0) <= SWEEP_TOL


@pytest.mark.parametrize("name", list(PROBS))
def test_q2_fgmres_parity(fc, oracles, name):
    p = PROBS[name]
    s = solver(fc, p)
    mg = oracles[name]
    b = mg.rhs()
    x_or, its_or, _ = mg.fgmres(b, rtol=1e-8)
    x, its, rr = s.solve(s.rhs(), rtol=1e-8)
    assert its == its_or and rr <= 1e-8
    assert rel(x.cpu().numpy(), x_or) <= 1e-6


def test_q2_standalone_gmg(fc):
    p = inputs.channel_replay_2d(0, nx=128, ny=32, nlevels=3)
    mg = O.Q2MG(p)
    b = mg.rhs()
    x_or, its_or, red_or = mg.gmg_solve(b, reduction=1e-9, maxit=80)
    s = solver(fc, p)
    x, its, red = s.gmg_solve(s.rhs(), reduction=1e-9, maxit=80)
    assert its == its_or and red <= 1e-9
    assert rel(x.cpu().numpy(), x_or) <= 1e-6


def test_q2_rejects_unsupported(fc):
    with pytest.raises(fc.FcError):
        fc.Solver(PROBS["ch2d"], element="q2", prec="df64")
    with pytest.raises(fc.FcError):
        fc.Solver(PROBS["por3d4"], element="q2", cache="matrix")
    s = solver(fc, PROBS["ch2d"])
    x = s.zeros()
    assert s.smooth_noalloc_(x, s.rhs()) == fc.FC_ERR_INVALID
