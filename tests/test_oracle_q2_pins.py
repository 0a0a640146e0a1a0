"""Pins of the Q2-Q1 (Taylor-Hood) oracle with the lower-corner ownership
rule, against what mathematics and the paper fix (CPU only).

- uncut element matrices: the textbook 1D Q2 stiffness and mass matrices
  (tensor products) and exactly integrated divergence couplings;
- quadrature: area and perimeter of the fluid region;
- ownership: every free DoF (each Q2 velocity node component and each
  pressure) is written by exactly one patch (Sec. 3.1, R~_i);
- local solves: a patch covering the whole grid turns one undamped sweep
  into the direct solve on the DoFs it owns; owned rows against a library
  solve of the equilibrated patch matrix;
- the sweep does not depend on the patch order (bitwise);
- transfers: Q2 interpolation is exact on quadratic velocities and Q1 on
  linear pressures (nested spaces), restriction is the transpose;
- discretisation: Taylor-Hood rates on uncut grids (velocity h^3, pressure
  h^2) for manufactured flows;
- solvers: FGMRES-GMG reaches the direct solution; iteration counts stay
  bounded as the grid is refined.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse.linalg as spl

from oracle import oracle as O
from paper_2403_11636_gb300 import inputs

ETA = 1e-3


def level(dim, n, shapes=None, alpha=1e-8, qdepth=3, preset=2, force_kind=0, force=(0, 0, 0), omega=0.8,
          ubar=0.3, hi=None):
    shapes = np.zeros((0, 9)) if shapes is None else shapes
    return O.Q2Level(dim, (n,) * dim, (0.0,) * dim, hi or (1.0,) * dim, shapes, alpha, qdepth, ETA, 100.0, omega,
                     preset, force_kind, force, ubar)


# ------------------------------------------------------------------ exact 1D
def q2_polys():
    """Q2 basis on [0, 1] as coefficient lists (ascending powers, exact)."""
    return [[Fraction(1), Fraction(-3), Fraction(2)],       # (1-t)(1-2t)
            [Fraction(0), Fraction(4), Fraction(-4)],       # 4t(1-t)
            [Fraction(0), Fraction(-1), Fraction(2)]]       # t(2t-1)


def q1_polys():
    return [[Fraction(1), Fraction(-1)], [Fraction(0), Fraction(1)]]


def pmul(a, b):
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def pder(a):
    return [a[k] * k for k in range(1, len(a))] or [Fraction(0)]


def pint01(a):
    return sum(c / (k + 1) for k, c in enumerate(a))


def one_d(h):
    """Exact 1D matrices on a cell of width h: Q2 stiffness K, Q2 mass M,
    Q2 derivative x Q1 G, Q2 x Q1 P, Q2 integrals m."""
    q, m = q2_polys(), q1_polys()
    K = np.array([[float(pint01(pmul(pder(a), pder(b)))) for b in q] for a in q]) / h
    M = np.array([[float(pint01(pmul(a, b))) for b in q] for a in q]) * h
    G = np.array([[float(pint01(pmul(pder(a), b))) for b in m] for a in q])
    P = np.array([[float(pint01(pmul(a, b))) for b in m] for a in q]) * h
    mi = np.array([float(pint01(a)) for a in q]) * h
    return K, M, G, P, mi


def test_one_d_matrices_are_the_textbook_ones():
    """Retyped from the textbook (Q2 Lagrange on [0, h]), independent of the
    exact integration above."""
    K, M, _, _, mi = one_d(1.0)
    np.testing.assert_allclose(K, np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / 3.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(M, np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) / 30.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(mi, [1 / 6, 2 / 3, 1 / 6], rtol=0, atol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_uncut_element_matrices_closed_form(dim):
    n = 4
    h = 1.0 / n
    L = level(dim, n, force_kind=0, force=(0.7, -0.3, 0.2))
    e = L.cell_element(5)
    K, M, G, P, mi = one_d(h)
    na = 3 ** dim
    ia = [(a % 3, (a // 3) % 3, a // 9) for a in range(na)]
    A = np.zeros((na, na))
    for a in range(na):
        for b in range(na):
            s = 0.0
            for k in range(dim):
                t = K[ia[a][k], ia[b][k]]
                for m in range(dim):
                    if m != k:
                        t *= M[ia[a][m], ia[b][m]]
                s += t
            A[a, b] = ETA * s
    np.testing.assert_allclose(e["A"], A, rtol=1e-12, atol=1e-14 * np.abs(A).max())
    # B_c[a][b] = -int d_c N_a M_b
    nb = 1 << dim
    for c in range(dim):
        Bc = np.zeros((na, nb))
        for a in range(na):
            for b in range(nb):
                t = -G[ia[a][c], (b >> c) & 1]
                for m in range(dim):
                    if m != c:
                        t *= P[ia[a][m], (b >> m) & 1]
                Bc[a, b] = t
        np.testing.assert_allclose(e["B"][c], Bc, rtol=1e-12, atol=1e-14 * np.abs(Bc).max())
    f = np.array([0.7, -0.3, 0.2])[:dim]
    for c in range(dim):
        want = np.array([f[c] * np.prod([mi[ia[a][k]] for k in range(dim)]) for a in range(na)])
        np.testing.assert_allclose(e["f"][c], want, rtol=1e-12)
    assert e["nbnd"] == 0


def test_cut_quadrature_area_and_perimeter():
    """A circle of radius 0.3: the fluid volumes sum to 1 - pi r^2 within
    the sub-cell error of the box split, the boundary weights to 2 pi r."""
    r = 0.3
    sh = np.array([[0.0, 0.5, 0.5, 0.0, r, r, r, 1.0, 0.0]])
    for k in (3, 4):
        L = level(2, 8, shapes=sh, qdepth=k)
        vol = sum(L.cell_element(c)["fluid_volume"] for c in range(L.ncell))
        per = sum(L.cell_element(c)["boundary_measure"] for c in range(L.ncell))
        assert abs(vol - (1 - math.pi * r * r)) < 0.2 * 2.0 ** -k * 2 * math.pi * r / 8
        assert abs(per - 2 * math.pi * r) < 1e-8


@pytest.mark.parametrize("dim", [2, 3])
def test_q2_nitsche_forms_on_linear_fields(dim):
    """For v = the Q2 interpolant of a linear field l = g.x + l0 (exact in
    Q2), the assembled a(v, v) equals its closed form: the alpha-weighted
    volume term plus -2(v, n.eta grad v)_G = 2 eta int (g.e)^2 and
    (v, lambda v)_G on the circle / sphere; b(v, 1) = -g_0 int alpha +
    int l n_0 (eq. stokes_disc_weak_fcm_2 with the symmetric Nitsche terms)."""
    n, r, alpha, beta = 8, 0.2, 1e-8, 100.0
    c = (0.47, 0.52, 0.49)
    sh = np.array([[0.0, c[0], c[1], c[2] if dim == 3 else 0.0, r, r, r, 1.0, 0.0]])
    L = level(dim, n, shapes=sh, alpha=alpha)
    A, _, _ = L.csr()
    g1 = np.linspace(0, 1, 2 * n + 1)
    P = [m.ravel() for m in np.meshgrid(*([g1] * dim), indexing="ij")[::-1]]   # x fastest
    g = np.array([0.7, -1.3, 0.4][:dim])
    l0 = 0.3
    v = np.zeros(L.ndof)
    v[0:L.nv:dim] = l0 + sum(g[k] * P[k] for k in range(dim))
    vf = sum(L.cell_element(cc)["fluid_volume"] for cc in range(L.ncell))
    lc = l0 + float(g @ np.array(c[:dim]))
    g2 = float(g @ g)
    lam = beta * ETA * n
    vol_term = ETA * g2 * (vf + alpha * (1 - vf))
    if dim == 2:
        exp = vol_term + 2 * ETA * math.pi * r * r * g2 + lam * r * math.pi * (2 * lc * lc + r * r * g2)
        bnd_b = -math.pi * r * r * g[0]
    else:
        exp = (vol_term + (8 * math.pi / 3) * ETA * r ** 3 * g2
               + lam * r * r * (4 * math.pi * lc * lc + r * r * (4 * math.pi / 3) * g2))
        bnd_b = -(4 * math.pi / 3) * r ** 3 * g[0]
    assert abs(v @ (A @ v) - exp) < 1e-10 * exp
    q = np.zeros(L.ndof)
    q[L.nv:] = 1.0
    expb = -g[0] * (vf + alpha * (1 - vf)) + bnd_b
    assert abs(v @ (A @ q) - expb) < 1e-10 * abs(expb)


# ----------------------------------------------------------------- ownership
@pytest.mark.parametrize("dim,preset", [(2, 0), (2, 1), (3, 1), (3, 0)])
def test_owner_count_is_one(dim, preset):
    n = 6 if dim == 2 else 4
    sh = np.array([[0.0, 0.4, 0.45, 0.5, 0.17, 0.17, 0.17, 1.0, 0.0]])
    L = level(dim, n, shapes=sh, preset=preset)
    _, _, fixed = L.csr()
    cnt = L.owner_count()
    assert np.all(cnt[~fixed] == 1)
    assert np.all(cnt[fixed] == 0)
    assert fixed[:L.nv].any() and not fixed[L.nv:].any()   # pressures are never constrained


@pytest.mark.parametrize("dim", [2, 3])
def test_whole_domain_patch_is_the_direct_solve(dim):
    """On a 2^d-cell grid the patch of the centre vertex holds every free
    DoF (L_i = L on the free DoFs), so one damped sweep from any x0 moves the
    DoFs it owns to x0 + omega (x* - x0) with x* the direct solution, and the
    Dirichlet DoFs to their values (identity rows)."""
    sh = np.array([[0.0, 0.4, 0.55, 0.5, 0.2, 0.2, 0.2, 1.0, 0.0]])
    L = level(dim, 2, shapes=sh, preset=0, omega=0.8, force_kind=0, force=(1.0, 0.5, 0.2))
    A, b, fixed = L.csr()
    centre = 1 + 3 * (1 + (3 if dim == 3 else 0))
    dofs, own = L.patch_dofs(centre)
    assert len(dofs) == int((~fixed).sum())
    x0 = inputs.uniform_array(L.ndof, 9)
    x1 = L.sweep(b, x0)
    xd = spl.spsolve(A.tocsc(), b)
    owned = dofs[own[own >= 0]]
    want = x0[owned] + 0.8 * (xd[owned] - x0[owned])
    np.testing.assert_allclose(x1[owned], want, rtol=1e-9, atol=1e-12 * np.abs(xd).max())
    np.testing.assert_allclose(x1[fixed], b[fixed], rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_q2_patch_sizes(dim):
    """Patch DoF counts (no constraints): an interior vertex holds the 9^d Q2
    nodes with d components each and 3^d pressures (171 in 2D, 2,214 in 3D)
    and owns 2^d d + 1 of them; the corner vertex keeps the 5^d Q2 nodes and
    2^d pressures inside the grid."""
    n = 6 if dim == 2 else 4
    L = level(dim, n)
    L.assemble()
    nv1 = n + 1
    interior = 3 + nv1 * (3 if dim == 2 else (2 + nv1 * 2))
    if dim == 3:
        interior = 2 + nv1 * (2 + nv1 * 2)
    dofs, own = L.patch_dofs(interior)
    assert len(dofs) == (9 ** dim) * dim + 3 ** dim
    assert (own >= 0).sum() == (1 << dim) * dim + 1
    dofs0, own0 = L.patch_dofs(0)
    assert len(dofs0) == (5 ** dim) * dim + 2 ** dim


@pytest.mark.parametrize("dim", [2, 3])
def test_owned_rows_match_a_library_solve(dim):
    n = 8 if dim == 2 else 4
    sh = np.array([[0.0, 0.45, 0.5, 0.5, 0.21, 0.21, 0.21, 1.0, 0.0]])
    L = level(dim, n, shapes=sh, preset=1)
    L.assemble()
    nv1 = n + 1
    verts = [nv1 * (n // 2) + n // 2, 0, nv1 * 3 + 2] if dim == 2 else [2 + nv1 * (2 + nv1 * 2), 1 + nv1 * 2]
    for v in verts:
        Li, dofs, own = L.patch_matrix(v)
        rows, dofs2, own2 = L.patch_inverse_rows(v)
        assert np.array_equal(dofs, dofs2)
        d = 1.0 / np.sqrt(np.abs(Li).max(axis=1))
        Ls = d[:, None] * Li * d[None, :]
        for k in np.where(own >= 0)[0]:
            e = np.zeros(len(dofs))
            e[own[k]] = 1.0
            z = d * np.linalg.solve(Ls, d * e)
            assert np.linalg.norm(rows[k] - z) <= 1e-10 * np.linalg.norm(z)


def test_sweep_order_independent_bitwise():
    p = inputs.channel_2d(0, n=16, nlevels=2)
    L = O.Q2Level.from_problem(p)
    x0 = inputs.uniform_array(L.ndof, 3)
    b = inputs.uniform_array(L.ndof, 4)
    a1 = L.sweep(b, x0)
    perm = np.random.default_rng(0).permutation(L.np)
    a2 = L.sweep(b, x0, order=perm)
    np.testing.assert_array_equal(a1, a2)


# ----------------------------------------------------------------- transfers
@pytest.mark.parametrize("dim", [2, 3])
def test_transfers_exact_and_transposed(dim):
    nc = 4 if dim == 2 else 2
    C = level(dim, nc)
    F = level(dim, 2 * nc)

    def q2_nodes(lv, n):
        g = np.linspace(0, 1, 2 * n + 1)
        mesh = np.meshgrid(*([g] * dim), indexing="ij")
        return [m.transpose().ravel() for m in mesh]   # x fastest

    def verts(n):
        g = np.linspace(0, 1, n + 1)
        mesh = np.meshgrid(*([g] * dim), indexing="ij")
        return [m.transpose().ravel() for m in mesh]

    def field(lv, n):
        X = q2_nodes(lv, n)
        u = np.zeros((len(X[0]), dim))
        for c in range(dim):
            u[:, c] = 1 + 2 * X[0] - X[1] ** 2 + 3 * X[0] * X[1] + (c + 1) * X[dim - 1] ** 2
        V = verts(n)
        p = 0.5 - V[0] + 2 * V[1] + (V[2] if dim == 3 else 0)
        return np.concatenate([u.ravel(), p])

    ec = field(C, nc)
    got = O.q2_prolong_add(F, C, ec, np.zeros(F.ndof))
    np.testing.assert_allclose(got, field(F, 2 * nc), rtol=0, atol=1e-13)
    rng = np.random.default_rng(1)
    rf = rng.standard_normal(F.ndof)
    e = rng.standard_normal(C.ndof)
    lhs = O.q2_restrict(F, C, rf) @ e
    rhs = rf @ O.q2_prolong_add(F, C, e, np.zeros(F.ndof))
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


# ---------------------------------------------------------- discretisation
def test_manufactured_2d_channel_rates():
    """Poiseuille flow u = (4 ubar y(1-y), 0) with p = 8 ubar eta (1-x) +
    s cos(pi x / 2) and the balancing force: uncut Taylor-Hood grids give a
    velocity error falling at least as h^2.5 (h^3 expected) and a pressure
    error as h^1.8 (h^2 expected); a velocity error at round-off counts as
    exact."""
    s, ubar = 0.01, 0.3
    eu, ep = [], []
    for n in (4, 8, 16):
        L = level(2, n, preset=0, force_kind=3, force=(s, 0, 0), ubar=ubar)
        A, b, _ = L.csr()
        x = spl.spsolve(A.tocsc(), b)
        u = x[:L.nv].reshape(2 * n + 1, 2 * n + 1, 2)
        g = np.linspace(0, 1, 2 * n + 1)
        Y, X = np.meshgrid(g, g, indexing="ij")
        eu.append(np.abs(u[:, :, 0] - 4 * ubar * Y * (1 - Y)).max() + np.abs(u[:, :, 1]).max())
        pv = x[L.nv:].reshape(n + 1, n + 1)
        gv = np.linspace(0, 1, n + 1)
        Yv, Xv = np.meshgrid(gv, gv, indexing="ij")
        ep.append(np.abs(pv - (8 * ubar * ETA * (1 - Xv) + s * np.cos(np.pi * Xv / 2))).max())
    for k in range(2):
        assert eu[k + 1] < 1e-11 or math.log2(eu[k] / eu[k + 1]) > 2.5
        assert math.log2(ep[k] / ep[k + 1]) > 1.8


def test_manufactured_3d_duct_rate():
    """u = (sin(pi y) sin(pi z), 0, 0), p = 0, f = (2 pi^2 eta sin sin, 0, 0)
    with no-slip y and z faces: velocity error at least h^2.5 (h^3
    expected)."""
    err = []
    for n in (2, 4, 8):
        L = level(3, n, preset=1, force_kind=2, force=(2 * math.pi ** 2 * ETA, 0, 0))
        A, b, _ = L.csr()
        x = spl.spsolve(A.tocsc(), b)
        u = x[:L.nv].reshape(2 * n + 1, 2 * n + 1, 2 * n + 1, 3)
        g = np.linspace(0, 1, 2 * n + 1)
        Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
        err.append(np.abs(u[..., 0] - np.sin(np.pi * Y) * np.sin(np.pi * Z)).max())
        assert np.abs(u[..., 1:]).max() < 1e-9
    for k in range(2):
        assert math.log2(err[k] / err[k + 1]) > 2.5


# ------------------------------------------------------------------ solvers
@pytest.mark.parametrize("dim", [2, 3])
def test_q2_fgmres_reaches_direct_solution(dim):
    p = inputs.channel_2d(0, n=16, nlevels=3) if dim == 2 else inputs.porous_3d(0, n=4, nspheres=2, nlevels=2)
    mg = O.Q2MG(p)
    A, b, _ = mg.fine.csr()
    x, its, rel = mg.fgmres(b, rtol=1e-10)
    xd = spl.spsolve(A.tocsc(), b)
    assert rel <= 1e-10 and its <= 40
    assert np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)


def test_q2_iteration_counts_bounded_under_refinement():
    its = []
    for n, nl in ((16, 2), (32, 3), (64, 4)):
        p = inputs.channel_2d(0, n=n, nlevels=nl)
        mg = O.Q2MG(p)
        _, k, rel = mg.fgmres(mg.rhs(), rtol=1e-8)
        assert rel <= 1e-8
        its.append(k)
    assert max(its) <= 2 * min(its) + 2, its
