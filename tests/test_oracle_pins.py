"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Nothing here calls the CUDA library.  Each test checks the oracle against an
independent fact: a textbook closed form, an exact integral, an invariant, a
value printed in the paper, a special case that reduces to a library solve,
or a high-precision (mpmath) solve.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spl

from oracle import oracle as O
from paper_2403_11636_gb300 import inputs

ETA = 1e-3
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def level(dim, n, shapes=None, alpha=1e-8, qdepth=None, preset=2, force_kind=0,
          force=(0.0, 0.0, 0.0), eta=ETA, omega=0.8, lo=None, hi=None):
    if shapes is None:
        shapes = np.zeros((0, 9))
    if qdepth is None:
        qdepth = 4 if dim == 2 else 3
    nn = (n,) * dim if isinstance(n, int) else n
    return O.Level(dim, nn, lo or (0.0,) * dim, hi or (1.0,) * dim, shapes, alpha, qdepth, eta,
                   100.0, omega, preset, force_kind, force, 0.3)


def circle(cx, cy, r):
    return np.array([[0.0, cx, cy, 0.0, r, r, r, 1.0, 0.0]])


def sphere(c, r):
    return np.array([[0.0, c[0], c[1], c[2], r, r, r, 1.0, 0.0]])


# ---------------------------------------------------------------- 1D textbook
def k1(h):   # 1D stiffness int phi_a' phi_b'
    return np.array([[1.0, -1.0], [-1.0, 1.0]]) / h


def m1(h):   # 1D mass int phi_a phi_b
    return np.array([[2.0, 1.0], [1.0, 2.0]]) * h / 6.0


def d1():    # 1D int phi_a' phi_b  (a: derivative, b: value)
    return np.array([[-0.5, -0.5], [0.5, 0.5]])


def kron_dims(mats):
    """Tensor product over directions with local index a = a_x + 2 a_y + 4 a_z."""
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(m, out)
    return out


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("fluid", [True, False])
def test_uncut_element_matrices_closed_form(dim, fluid):
    """Q1 element matrices of an uncut cell equal the tensor-product textbook
    forms: a = eta*alpha*K, b_c = -alpha*(D in direction c, M elsewhere),
    c = -(1/eta)(M - m m^T/|K|) without alpha (Sec. 2, eq. stokes_disc_weak_fcm_2,
    eq. stabilization_l2), f = alpha F |K| / 2^d."""
    n = 4
    h = 1.0 / n
    alpha = 1e-6
    # obstacle covering everything (fictitious) or nothing (fluid)
    sh = (circle(0.5, 0.5, 5.0) if dim == 2 else sphere((0.5, 0.5, 0.5), 5.0)) if not fluid else None
    F = (0.7, -0.2, 0.4)
    L = level(dim, n, sh, alpha=alpha, force_kind=0, force=F)
    e = L.cell_element(5)
    a = 1.0 if fluid else alpha
    K = sum(kron_dims([k1(h) if k == j else m1(h) for k in range(dim)]) for j in range(dim))
    np.testing.assert_allclose(e["A"], ETA * a * K, rtol=1e-13, atol=1e-13 * ETA * a)
    for c in range(dim):
        Bc = -a * kron_dims([d1() * (1.0 if k == c else 0.0) + (m1(h) if k != c else 0.0)
                             for k in range(dim)])
        np.testing.assert_allclose(e["B"][c], Bc, rtol=1e-13, atol=1e-15)
    M = kron_dims([m1(h)] * dim)
    vol = h ** dim
    m = np.full(2 ** dim, vol / 2 ** dim)
    np.testing.assert_allclose(e["C"], -(M - np.outer(m, m) / vol) / ETA, rtol=1e-13, atol=1e-16)
    for c in range(dim):
        np.testing.assert_allclose(e["f"][c], a * F[c] * vol / 2 ** dim, rtol=1e-13, atol=1e-18)
    assert e["nbnd"] == 0


def test_textbook_2d_laplacian_numbers():
    """The unit-square Q1 Laplacian is (1/6)[[4,-1,-1,-2],...] (any h in 2D)."""
    L = level(2, 8, None)
    e = L.cell_element(0)
    ref = np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6.0
    np.testing.assert_allclose(e["A"] / ETA, ref, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_stabilisation_annihilates_constants(dim):
    """c(q, 1) = 0 for every q (q - Pi0 q has zero cell mean), c is symmetric
    negative semidefinite with a one-dimensional kernel per cell."""
    L = level(dim, 4, circle(0.5, 0.5, 0.3) if dim == 2 else sphere((0.5, 0.5, 0.5), 0.3))
    for cell in (0, 7, 13 if dim == 2 else 21):
        Cm = L.cell_element(cell)["C"]
        np.testing.assert_allclose(Cm.sum(axis=1), 0.0, atol=1e-14 * np.abs(Cm).max())
        np.testing.assert_array_equal(Cm, Cm.T)
        ev = np.linalg.eigvalsh(Cm)
        assert ev.max() <= 1e-12 * np.abs(ev).max()
        assert np.sum(np.abs(ev) < 1e-12 * np.abs(ev).max()) == 1


# ---------------------------------------------------------------- quadrature
@pytest.mark.parametrize("dim", [2, 3])
def test_fluid_volume_converges_with_depth(dim):
    """The recursive cut-cell rule gives the fluid measure 1 - |obstacle|, with
    an error that falls as the quadtree/octree depth grows."""
    n = 8
    r = 0.23
    c = (0.47, 0.52, 0.49)
    sh = circle(c[0], c[1], r) if dim == 2 else sphere(c, r)
    exact = 1.0 - (math.pi * r * r if dim == 2 else 4.0 / 3.0 * math.pi * r ** 3)
    errs = []
    depths = (1, 2, 3, 4, 5) if dim == 2 else (1, 2, 3)
    for k in depths:
        L = level(dim, n, sh, qdepth=k)
        vf = sum(L.cell_element(cc)["fluid_volume"] for cc in range(L.ncell))
        errs.append(abs(vf - exact))
    # error bound: boundary measure times the leaf size
    perim = 2 * math.pi * r if dim == 2 else 4 * math.pi * r * r
    for k, e in zip(depths, errs):
        assert e < perim * (1.0 / n) / 2 ** k
    assert errs[-1] < errs[0] / 4


def test_ellipse_area():
    """The level set of a rotated ellipse encloses pi a b (fluid = 1 - pi a b)."""
    a, b, th = 0.21, 0.09, 0.6
    sh = np.array([[1.0, 0.47, 0.52, 0.0, a, b, 0.0, math.cos(th), math.sin(th)]])
    L = level(2, 16, sh, qdepth=5)
    vf = sum(L.cell_element(cc)["fluid_volume"] for cc in range(L.ncell))
    assert abs(vf - (1.0 - math.pi * a * b)) < 2 * math.pi * a * (1.0 / 16) / 2 ** 5


def test_overlapping_obstacles_form_a_union():
    """Several obstacles: the fictitious part is the union of the shapes
    (phi = max over shapes, Sec. 2), and the boundary rule keeps only the
    parts of each curve outside the other obstacles, so the fluid measure is
    1 - |union| and the boundary weights add up to the union's perimeter.  Two
    circles of radius r at distance d < 2 r: |union| = 2 pi r^2 - lens,
    lens = 2 r^2 acos(d / 2r) - (d / 2) sqrt(4 r^2 - d^2), perimeter
    4 r (pi - acos(d / 2r))."""
    r, c1, c2 = 0.18, (0.40, 0.50), (0.62, 0.52)
    d = math.hypot(c2[0] - c1[0], c2[1] - c1[1])
    th = math.acos(d / (2 * r))
    union = 2 * math.pi * r * r - (2 * r * r * th - 0.5 * d * math.sqrt(4 * r * r - d * d))
    perim = 4 * r * (math.pi - th)
    n, k = 16, 5
    L = level(2, n, np.vstack([circle(*c1, r), circle(*c2, r)]), qdepth=k)
    vf = sum(L.cell_element(cc)["fluid_volume"] for cc in range(L.ncell))
    assert abs(vf - (1.0 - union)) < perim * (1.0 / n) / 2 ** k
    x, nrm, w, cell = L.bpoints()
    # four rule intervals straddle the two intersection points at most
    npts = 8 * math.ceil(2 * math.pi * r * n) * 2 ** k
    assert abs(w.sum() - perim) <= 4 * (2 * math.pi * r / npts)
    # divergence theorem over the union, n pointing out of the fluid
    xn = (w * ((x[:, :2] - np.array(c1)) * nrm[:, :2]).sum(axis=1)).sum()
    assert abs(xn + 2 * union) < 4 * (2 * math.pi * r / npts) * 2 * r


@pytest.mark.parametrize("dim,preset", [(2, 0), (2, 1), (3, 0), (3, 1)])
def test_presets_constrain_the_faces_of_the_setups(dim, preset):
    """Strong Dirichlet data of the two setups (Sec. 4): no-slip velocity on
    the walls y = lo, hi (and z = lo, hi), and for the channel also the
    inflow face x = lo; the outflow face x = hi stays free (natural
    condition) and the pressure is never constrained.  Wall values are zero."""
    n = 6
    L = level(dim, n, None, preset=preset)
    L.assemble()
    _, rhs, fixed = L.csr()
    nd = dim + 1
    idx = np.indices((n + 1,) * dim).reshape(dim, -1)[::-1]   # x fastest
    wall = (idx[1] == 0) | (idx[1] == n)
    if dim == 3:
        wall |= (idx[2] == 0) | (idx[2] == n)
    want = wall | (idx[0] == 0) if preset == 0 else wall
    fixed = fixed.reshape(-1, nd)
    for c in range(dim):
        np.testing.assert_array_equal(fixed[:, c], want)
    assert not fixed[:, dim].any()
    assert np.all(rhs.reshape(-1, nd)[wall, :dim] == 0.0)


def test_load_vector_channel_force():
    """f(v) = (v, alpha f) for f = (sin(pi x), cos(pi y)) on an uncut cell
    equals an adaptive 2D quadrature of f_c times the Q1 nodal function."""
    import scipy.integrate as si
    n = 16
    h = 1.0 / n
    L = level(2, n, None, force_kind=1, force=(1.0, 1.0, 0.0))
    cell = 5 + 16 * 9
    i, j = cell % n, cell // n
    e = L.cell_element(cell)
    for a in range(4):
        ax, ay = a & 1, a >> 1
        def phi(y, x):
            xi, et = (x - i * h) / h, (y - j * h) / h
            return (xi if ax else 1 - xi) * (et if ay else 1 - et)
        fx = si.dblquad(lambda y, x: math.sin(math.pi * x) * phi(y, x), i * h, (i + 1) * h,
                        j * h, (j + 1) * h, epsabs=1e-14)[0]
        fy = si.dblquad(lambda y, x: math.cos(math.pi * y) * phi(y, x), i * h, (i + 1) * h,
                        j * h, (j + 1) * h, epsabs=1e-14)[0]
        # the 2-point Gauss rule is exact to degree 3; sin/cos on a cell of
        # size h are integrated to O(h^4) relative accuracy
        assert abs(e["f"][0][a] - fx) < 1e-4 * abs(fx) + 1e-12
        assert abs(e["f"][1][a] - fy) < 1e-4 * abs(fy) + 1e-12


@pytest.mark.parametrize("dim,shape", [(2, "circle"), (2, "ellipse"), (3, "sphere")])
def test_boundary_rule_exact_integrals(dim, shape):
    """Sum of weights = perimeter / surface area; sum w n = 0 for a closed
    curve/surface; sum w (x - c).n = -d |obstacle| (divergence theorem, n
    pointing into the obstacle, i.e. out of the fluid)."""
    c = np.array([0.47, 0.52, 0.49])
    if shape == "circle":
        r = 0.2
        sh = circle(c[0], c[1], r)
        meas, vol = 2 * math.pi * r, math.pi * r * r
    elif shape == "ellipse":
        a, b, th = 0.21, 0.09, 0.6
        sh = np.array([[1.0, c[0], c[1], 0.0, a, b, 0.0, math.cos(th), math.sin(th)]])
        import scipy.special as ss
        meas = 4 * a * ss.ellipe(1 - (b / a) ** 2)
        vol = math.pi * a * b
    else:
        r = 0.2
        sh = sphere(c, r)
        meas, vol = 4 * math.pi * r * r, 4.0 / 3.0 * math.pi * r ** 3
    L = level(dim, 8, sh)
    x, nrm, w, cell = L.bpoints()
    assert abs(w.sum() - meas) < 1e-12 * meas
    np.testing.assert_allclose((w[:, None] * nrm).sum(axis=0), 0.0, atol=1e-13)
    xn = (w * ((x - c) * nrm)[:, :dim].sum(axis=1)).sum()
    assert abs(xn + dim * vol) < 1e-12 * vol
    # every point lies on the curve / surface and in the cell it is binned to
    h = 1.0 / 8
    idx = np.floor(x[:, :dim] / h).astype(int).clip(0, 7)
    lin = idx[:, 0] + 8 * idx[:, 1] + (64 * idx[:, 2] if dim == 3 else 0)
    np.testing.assert_array_equal(lin, cell)


@pytest.mark.parametrize("dim", [2, 3])
def test_nitsche_forms_on_linear_fields(dim):
    """For v = u = the Q1 interpolant of a linear field l = g.x + l0 (exact in
    Q1), the assembled a(v, v) equals its closed form: the alpha-weighted
    volume term plus -2(v, n.eta grad v)_G = 2 eta int (g.e)^2 and
    (v, lambda v)_G on the circle/sphere; b(v, 1) = -g_0 int alpha
    + int l n_0 (Sec. 2, eq. stokes_disc_weak_fcm_2)."""
    n, r, alpha, beta = 16, 0.2, 1e-8, 100.0
    c = (0.47, 0.52, 0.49)
    sh = circle(c[0], c[1], r) if dim == 2 else sphere(c, r)
    L = level(dim, n, sh, alpha=alpha)
    A, _, _ = L.csr()
    nd = dim + 1
    xs = np.linspace(0, 1, n + 1)
    grids = np.meshgrid(*([xs] * dim), indexing="ij")[::-1]   # x fastest
    P = [gg.ravel() for gg in grids]
    g = np.array([0.7, -1.3, 0.4][:dim])
    l0 = 0.3
    v = np.zeros(L.ndof)
    v[0::nd] = l0 + sum(g[k] * P[k] for k in range(dim))
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
    q[dim::nd] = 1.0
    expb = -g[0] * (vf + alpha * (1 - vf)) + bnd_b
    assert abs(v @ (A @ q) - expb) < 1e-10 * abs(expb)


# ---------------------------------------------------------------- operator
def test_dof_count_matches_paper_table():
    """Table tab:grid, Omega^1: 262,144 cells and 790,275 DoFs (Q1-Q1, 2D)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table_grid.txt")) if l.strip() and l[0] != "#"]
    nx, ny, cells, dofs = (int(t) for t in rows[0])
    L = level(2, (nx, ny), None, lo=(0.0, 0.0), hi=(2.2, 0.41))
    assert L.ncell == cells
    assert L.ndof == dofs


@pytest.mark.parametrize("dim,preset", [(2, 0), (2, 1), (3, 1), (3, 0)])
def test_operator_exactly_symmetric(dim, preset):
    """L is symmetric (symmetric Nitsche, B and B^T from one form, symmetric
    elimination of strong Dirichlet DoFs) -- bit for bit."""
    p = inputs.channel_2d(3, n=8) if dim == 2 else inputs.porous_3d(1, n=4, nspheres=3, nlevels=1)
    L = level(dim, 8 if dim == 2 else 4, p.shapes, alpha=p.alpha, preset=preset)
    A, b, fixed = L.csr()
    D = (A - A.T).tocoo()
    assert np.all(D.data == 0.0)
    # constrained rows are identity rows
    Ad = A.tocsr()
    for k in np.nonzero(fixed)[0][:50]:
        row = Ad.getrow(k)
        assert row.nnz == 0 or (np.count_nonzero(row.data) == 1 and Ad[k, k] == 1.0)


# ---------------------------------------------------------------- patches and sweep
def test_patch_sizes():
    """Interior patch: 5^d velocity nodes x d + 3^d pressure DoFs = 59 / 402
    (Sec. 3.1 definition of S_i with the structural reading)."""
    L2 = level(2, 8, None, preset=2)
    d, own = L2.patch_dofs(4 + 9 * 4)
    assert len(d) == 59 and list(own[:3]) == [24, 25, 54]
    L3 = level(3, 6, None, preset=2)
    node = 3 + 7 * 3 + 49 * 3
    d, own = L3.patch_dofs(node)
    assert len(d) == 402 and list(own) == [186, 187, 188, 388]


@pytest.mark.parametrize("dim", [2, 3])
def test_owner_count_is_one(dim):
    """Restricted prolongation: every free DoF is written by exactly one patch,
    constrained DoFs by none (Sec. 3.1, Sec. 3.1.1)."""
    p = inputs.channel_2d(1, n=8) if dim == 2 else inputs.porous_3d(2, n=4, nspheres=3, nlevels=1)
    L = O.Level.from_problem(p)
    _, _, fixed = L.csr()
    cnt = L.owner_count()
    np.testing.assert_array_equal(cnt[~fixed], 1)
    np.testing.assert_array_equal(cnt[fixed], 0)


def test_local_solves_exact_against_mpmath():
    """The owned rows of L_i^{-1} agree with a 40-digit solve of the same block
    on cut patches with alpha = 1e-8 (the LU reaches machine accuracy,
    Sec. 3.1.2)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    p = inputs.channel_2d(0, n=16, nlevels=1)
    L = O.Level.from_problem(p)
    L.assemble()
    rng = np.random.default_rng(0)
    checked = 0
    for node in rng.choice(L.nnodes, 12, replace=False):
        Li, dofs, own = L.patch_matrix(int(node))
        rows, d2, own2 = L.patch_inverse_rows(int(node))
        np.testing.assert_array_equal(dofs, d2)
        M = mpmath.matrix(Li.tolist())
        for c in range(3):
            if own[c] < 0:
                continue
            e = mpmath.matrix([1.0 if j == own[c] else 0.0 for j in range(len(dofs))])
            z = np.array([float(t) for t in mpmath.lu_solve(M, e)])
            assert np.linalg.norm(rows[c] - z) <= 1e-12 * np.linalg.norm(z)
            checked += 1
    assert checked >= 24


@pytest.mark.parametrize("dim", [2, 3])
def test_whole_domain_patch_is_exact_solve(dim):
    """On a one-cell grid every patch holds every DoF, so S = omega L^{-1} and
    one sweep with omega = 1 gives L^{-1} b from any x0 (eq. iteration)."""
    sh = circle(0.45, 0.55, 0.3) if dim == 2 else sphere((0.45, 0.55, 0.5), 0.3)
    L = level(dim, 1, sh, alpha=1e-6, omega=1.0, force_kind=0, force=(1.0, 0.5, 0.2))
    A, b, fixed = L.csr()
    x0 = inputs.uniform_array(L.ndof, 7)
    x1 = L.sweep(b, x0, mode=0)
    xd = np.linalg.solve(A.toarray(), b)
    assert np.linalg.norm(x1 - xd) <= 1e-11 * np.linalg.norm(xd)


@pytest.mark.parametrize("dim", [2, 3])
def test_sweep_order_and_partition_independent(dim):
    """The corrections are additive against one residual (Sec. 3.1.1): any
    patch order, or any split of the patches into groups applied one after
    the other against the frozen residual, gives bit-identical results."""
    p = inputs.channel_2d(2, n=8) if dim == 2 else inputs.porous_3d(3, n=4, nspheres=3, nlevels=1)
    L = O.Level.from_problem(p)
    A, b, fixed = L.csr()
    x0 = inputs.random_vector(p, 11)
    ref = L.sweep(b, x0, mode=0)
    perm = np.random.default_rng(1).permutation(L.nnodes)
    np.testing.assert_array_equal(L.sweep(b, x0, mode=0, order=perm), ref)
    r = L.residual(b, x0)
    x = x0.copy()
    for grp in np.array_split(perm, 5):
        x = L.apply_patches(r, x, grp)
    x[fixed] = x0[fixed] + r[fixed]
    np.testing.assert_array_equal(x, ref)


@pytest.mark.parametrize("dim", [2, 3])
def test_cached_inverse_equals_on_the_fly_solve(dim):
    """cache_inverse (stored owned rows) and gather-factor-solve per
    application give the same sweep up to rounding (Sec. 3.1.2)."""
    p = inputs.channel_2d(4, n=16) if dim == 2 else inputs.porous_3d(4, n=4, nspheres=4, nlevels=1)
    L = O.Level.from_problem(p)
    _, b, _ = L.csr()
    x0 = inputs.random_vector(p, 3)
    a = L.sweep(b, x0, mode=0)
    c = L.sweep(b, x0, mode=1)
    assert np.linalg.norm(a - c) <= 1e-13 * np.linalg.norm(a)


# ---------------------------------------------------------------- transfers
@pytest.mark.parametrize("dim", [2, 3])
def test_prolongation_exact_on_linear_fields(dim):
    """Q1 interpolation reproduces fields linear in x (every component)."""
    nc = 4
    C = level(dim, nc, None, preset=2)
    F = level(dim, 2 * nc, None, preset=2)
    def lin(n, coef):
        xs = np.linspace(0, 1, n + 1)
        grids = np.meshgrid(*([xs] * dim), indexing="ij")[::-1]
        v = np.zeros(((n + 1) ** dim, dim + 1))
        for c in range(dim + 1):
            v[:, c] = coef[c][0] + sum(coef[c][1 + k] * grids[k].ravel() for k in range(dim))
        return v.ravel()
    coef = np.random.default_rng(2).normal(size=(dim + 1, dim + 1))
    xf = O.prolong_add(F, C, lin(nc, coef), np.zeros(F.ndof))
    np.testing.assert_allclose(xf, lin(2 * nc, coef), rtol=0, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_restriction_is_transpose_of_prolongation(dim):
    """R = P^T (eq. restriction_op, P = R^T): <R r, e> = <r, P e>."""
    C = level(dim, 4, None, preset=2)
    F = level(dim, 8, None, preset=2)
    r = inputs.uniform_array(F.ndof, 5)
    e = inputs.uniform_array(C.ndof, 6)
    lhs = O.restrict(F, C, r) @ e
    rhs = r @ O.prolong_add(F, C, e, np.zeros(F.ndof))
    assert abs(lhs - rhs) <= 1e-13 * (np.abs(r).sum())


@pytest.mark.parametrize("dim,preset", [(2, 0), (2, 1), (3, 0), (3, 1)])
def test_restriction_with_strong_dirichlet_rows(dim, preset):
    """With strong Dirichlet data the coarse correction lives in the space of
    coarse functions that vanish on the constrained DoFs (Sec. 3): R r is
    exactly zero there, and on the free DoFs R = P^T for every fine residual
    that vanishes on the constrained fine DoFs (a smoothed residual, whose
    identity rows are satisfied): <R r, e> = <r, P e> for every coarse e that
    vanishes on the constrained coarse DoFs."""
    C = level(dim, 4, None, preset=preset)
    F = level(dim, 8, None, preset=preset)
    C.assemble()
    F.assemble()
    fixc, fixf = C.csr()[2], F.csr()[2]
    assert fixc.any() and fixf.any() and not fixc.all()
    r = inputs.uniform_array(F.ndof, 7)
    r[fixf] = 0.0
    e = inputs.uniform_array(C.ndof, 8)
    e[fixc] = 0.0
    rc = O.restrict(F, C, r)
    assert np.all(rc[fixc] == 0.0)
    assert np.any(rc[~fixc] != 0.0)
    lhs = rc @ e
    rhs = r @ O.prolong_add(F, C, e, np.zeros(F.ndof))
    assert abs(lhs - rhs) <= 1e-13 * (np.abs(r).sum())


# ---------------------------------------------------------------- discretisation
def test_manufactured_2d_channel_convergence():
    """Poiseuille flow plus a pressure field balanced by the body force,
    u = (4 ubar y(1-y), 0), p = 8 ubar eta (1-x) + s cos(pi x / 2), satisfies
    the channel boundary conditions exactly; on uncut grids the nodal
    velocity error falls as h^2 and the pressure error as h."""
    s, ubar = 0.01, 0.3
    eu, ep = [], []
    for n in (8, 16, 32):
        L = O.Level(2, (n, n), (0, 0), (1, 1), np.zeros((0, 9)), 1e-8, 4, ETA, 100.0, 0.8, 0, 3,
                    (s, 0, 0), ubar)
        A, b, _ = L.csr()
        x = spl.spsolve(A.tocsc(), b).reshape(n + 1, n + 1, 3)
        xs = np.linspace(0, 1, n + 1)
        Y, X = np.meshgrid(xs, xs, indexing="ij")
        eu.append(np.abs(x[:, :, 0] - 4 * ubar * Y * (1 - Y)).max())
        ep.append(np.abs(x[:, :, 2] - (8 * ubar * ETA * (1 - X) + s * np.cos(np.pi * X / 2))).max())
    for k in range(2):
        assert math.log2(eu[k] / eu[k + 1]) > 1.9
        assert math.log2(ep[k] / ep[k + 1]) > 0.9


def test_manufactured_3d_duct_convergence():
    """u = (sin(pi y) sin(pi z), 0, 0), p = 0 with f = (2 pi^2 eta sin sin, 0, 0)
    in the porous-preset box: velocity error falls as h^2, p stays 0."""
    err = []
    for n in (4, 8, 16):
        L = O.Level(3, (n,) * 3, (0,) * 3, (1,) * 3, np.zeros((0, 9)), 1e-8, 3, ETA, 100.0, 0.8, 1,
                    2, (2 * math.pi ** 2 * ETA, 0, 0), 0.3)
        A, b, _ = L.csr()
        x = spl.spsolve(A.tocsc(), b).reshape(n + 1, n + 1, n + 1, 4)
        xs = np.linspace(0, 1, n + 1)
        Z, Y, X = np.meshgrid(xs, xs, xs, indexing="ij")
        err.append(np.abs(x[..., 0] - np.sin(np.pi * Y) * np.sin(np.pi * Z)).max())
        assert np.abs(x[..., 1:]).max() < 1e-10
    for k in range(2):
        assert math.log2(err[k] / err[k + 1]) > 1.9


# ---------------------------------------------------------------- solvers
@pytest.mark.parametrize("dim", [2, 3])
def test_fgmres_reaches_direct_solution(dim):
    """FGMRES with the GMG V-cycle as right preconditioner reaches the direct
    solution of the assembled system to the requested tolerance."""
    p = inputs.channel_2d(0, n=16, nlevels=2) if dim == 2 else inputs.porous_3d(0, n=8, nspheres=4, nlevels=2)
    mg = O.MG(p)
    A, b, _ = mg.fine.csr()
    x, its, rel, hist = mg.fgmres(b, rtol=1e-10)
    xd = spl.spsolve(A.tocsc(), b)
    assert rel <= 1e-10
    assert np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)
    assert its <= 30
    assert np.all(np.diff(hist) <= 1e-14)


def test_fgmres_exact_in_n_steps_without_preconditioner_effect():
    """With a direct coarse solve on a one-level hierarchy the preconditioner
    is L^{-1} and FGMRES converges in one step."""
    p = inputs.channel_2d(0, n=8, nlevels=1)
    mg = O.MG(p)
    x, its, rel, _ = mg.fgmres(mg.rhs(), rtol=1e-12)
    assert its == 1 and rel < 1e-12


def test_iteration_counts_bounded_under_refinement():
    """Iteration counts stay bounded as the grid is refined with a fixed
    coarsest grid of 8^2 cells (Sec. 4, mesh study)."""
    counts = []
    for n, nlev in ((16, 2), (32, 3), (64, 4), (128, 5)):
        p = inputs.channel_2d(0, n=n, nlevels=nlev)
        mg = O.MG(p)
        _, its, rel, _ = mg.fgmres(mg.rhs(), rtol=1e-8)
        assert rel <= 1e-8
        counts.append(its)
    assert max(counts) <= 16


def test_iteration_counts_h_independent_without_obstacle():
    """Without cut cells the V-cycle is a textbook GMG for the stabilised
    Q1-Q1 Stokes system and its FGMRES count does not grow with the depth of
    the hierarchy (fixed 8^2 coarsest grid)."""
    counts = []
    for n, nlev in ((16, 2), (32, 3), (64, 4), (128, 5)):
        p = inputs.channel_2d(0, n=n, nlevels=nlev)
        p.shapes = np.zeros((0, 9))
        mg = O.MG(p)
        _, its, rel, _ = mg.fgmres(mg.rhs(), rtol=1e-8)
        assert rel <= 1e-8
        counts.append(its)
    assert max(counts) - min(counts) <= 1


def test_standalone_gmg_reduces_residual():
    """Standalone GMG with V(6,6) and damping 0.8 reaches a 1e9 reduction
    (Sec. 4 solver setting)."""
    p = inputs.channel_2d(0, n=32, nlevels=3, alpha=1e-10)
    p.nu_pre = p.nu_post = 6
    mg = O.MG(p)
    _, its, red = mg.gmg_solve(mg.rhs(), reduction=1e-9, maxit=60)
    assert red <= 1e-9
    assert its <= 40


def _blocks(A, dim):
    nd = dim + 1
    v = np.array([k % nd < dim for k in range(A.shape[0])])
    A = A.toarray()
    return A[np.ix_(v, v)], A[np.ix_(v, ~v)], A[np.ix_(~v, v)], A[np.ix_(~v, ~v)]


@pytest.mark.parametrize("dim", [2, 3])
def test_galerkin_equals_rediscretisation_without_obstacles(dim):
    """Galerkin coarse operator R L_f P (the alternative to rediscretising the
    coarser grids, Sec. 3) on a grid without obstacles: the Q1 spaces are
    nested and the Gauss rule integrates the velocity and divergence forms
    exactly, so those blocks equal the rediscretised coarse operator,
    constrained wall and inflow rows included; the pressure block (a
    projection on each cell, which does not nest) does not."""
    if dim == 2:
        p = inputs.channel_2d(0, n=8, nlevels=2)
    else:
        p = inputs.porous_3d(0, n=4, nspheres=1, nlevels=2)
        p.preset = 0
    p.shapes = np.zeros((0, 9))
    gal = O.MG(p, galerkin=True).levels[0].csr()[0]
    red = O.Level.from_problem(p, 1).csr()[0]
    g, r = _blocks(gal, dim), _blocks(red, dim)
    for k in range(3):
        assert np.abs(g[k] - r[k]).max() <= 1e-12 * np.abs(r[k]).max(), k
    assert np.abs(g[3] - r[3]).max() >= 0.1 * np.abs(r[3]).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_galerkin_pressure_block_closed_form(dim):
    """The Galerkin pressure block applies the fine-grid stabilisation
    c(q,p) = -(1/eta) sum over fine cells K of |K| var_K(p) (eq.
    stabilization_l2) to coarse Q1 functions: it vanishes on constants, and
    for p = x it equals -(1/eta) |Omega| h_f^2 / 12 (the variance of a
    linear function over a cell of width h_f), a quarter of the rediscretised
    coarse value."""
    n = 8 if dim == 2 else 4
    if dim == 2:
        p = inputs.channel_2d(0, n=n, nlevels=2)
    else:
        p = inputs.porous_3d(0, n=n, nspheres=1, nlevels=2)
    p.shapes = np.zeros((0, 9))
    Cg = _blocks(O.MG(p, galerkin=True).levels[0].csr()[0], dim)[3]
    Cr = _blocks(O.Level.from_problem(p, 1).csr()[0], dim)[3]
    nc = n // 2
    xs = np.array([(k % (nc + 1)) / nc for k in range((nc + 1) ** dim)])
    assert np.abs(Cg @ np.ones(len(xs))).max() <= 1e-12 * np.abs(Cg).max()
    hf = 1.0 / n
    want = -(1.0 / p.eta) * hf * hf / 12.0
    assert xs @ Cg @ xs == pytest.approx(want, rel=1e-12)
    assert xs @ Cr @ xs == pytest.approx(4.0 * want, rel=1e-12)


def test_galerkin_hierarchy_converges():
    """FGMRES with Galerkin coarse operators on the channel with a cut
    circle reaches the direct solution within the rediscretised hierarchy's
    iteration bound (Sec. 4 solver setting)."""
    p = inputs.channel_2d(0, n=32, nlevels=3)
    mg = O.MG(p, galerkin=True)
    A, b, _ = mg.fine.csr()
    x, its, rel, _ = mg.fgmres(b, rtol=1e-10)
    assert rel <= 1e-10
    xd = spl.spsolve(A.tocsc(), b)
    assert np.linalg.norm(x - xd) <= 1e-7 * np.linalg.norm(xd)
    assert its <= 16
