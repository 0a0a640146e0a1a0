"""Pins of the adaptive-grid oracle (oracle/fc_oracle_amr.c): 2D quadtree
grids refined towards the obstacle boundary with 2:1 balance, hanging nodes
removed as constraints, and the hierarchy of Algorithm 1 (Sec. 3).

Each pin ties the adaptive construction to something fixed independently of
it: the uniform oracle (a tree refined uniformly is the uniform grid), the
balance and coarsening rules checked cell by cell on the level map, the
hanging-node geometry, exactness of the prolongation on linear fields, the
conforming finite element space (the adaptive bilinear forms equal those of
the uniform finest grid on the interpolated functions), and convergence of
FGMRES to the direct solution."""
import dataclasses

import numpy as np
import pytest
import scipy.sparse.linalg as spl

from oracle import oracle as O
from paper_2403_11636_gb300 import inputs


def channel(n=64, nlevels=4, u=1, alpha=1e-8):
    p = inputs.channel_2d(0, n=n, nlevels=nlevels, alpha=alpha)
    return dataclasses.replace(p, amr_uniform=u)


@pytest.fixture(scope="module")
def amr():
    p = channel()
    return p, O.amr_levels(p)


def test_uniform_tree_is_the_uniform_grid():
    p = dataclasses.replace(inputs.channel_2d(0, n=16, nlevels=3), amr_uniform=2)
    lv = O.amr_levels(p)
    for l in (1, 2, 3):
        A, b, f = lv[l - 1].csr()
        U = O.Level.from_problem(p, l)
        Au, bu, fu = U.csr()
        assert abs(A - Au).max() <= 1e-13 * abs(Au).max()
        assert np.abs(b - bu).max() <= 1e-13 * max(np.abs(bu).max(), 1.0)
        assert np.array_equal(f, fu)
        U.assemble()
        for node in (0, U.nnodes // 3, U.nnodes // 2, U.nnodes - 1):
            dofs = np.zeros(O.PMAX, dtype=np.int64); ow = np.zeros(O.OMAX, dtype=np.int32)
            n = U.lib.or_patch_dofs(U.h, node, O._p(dofs, O.C.c_long), O._p(ow, O.C.c_int))
            d2, own2 = lv[l - 1].patch_dofs(node)
            assert np.array_equal(dofs[:n], d2) and np.array_equal(ow, own2)
    # prolongation equals the uniform Q1 interpolation
    F, Cc = lv[2], lv[1]
    UF, UC = O.Level.from_problem(p, 3), O.Level.from_problem(p, 2)
    UF.assemble(); UC.assemble()
    e = inputs.uniform_array(Cc.ndof, 5)
    x = inputs.uniform_array(F.ndof, 6)
    assert np.abs(O.prolong_add(F, Cc, e, x) - O.prolong_add(UF, UC, e, x)).max() <= 1e-15


def test_refinement_balance_and_algorithm_1(amr):
    p, lv = amr
    R = p.nlevels - 1
    maps = [l.leaf_levels() for l in lv]
    fine = maps[-1]
    # cut leaves (sign change among the 3x3 sample points) are at the finest level
    G = O.Level.from_problem(dataclasses.replace(p, amr_uniform=-1))
    ny, nx = fine.shape
    hx, hy = (p.hi[0] - p.lo[0]) / nx, (p.hi[1] - p.lo[1]) / ny
    for Y in range(ny):
        for X in range(nx):
            l = fine[Y, X]
            s = 1 << (R - l)
            if X % s or Y % s:
                continue
            signs = set()
            for j in range(3):
                for i in range(3):
                    x = (O.C.c_double * 3)(p.lo[0] + (X + 0.5 * i * s) * hx, p.lo[1] + (Y + 0.5 * j * s) * hy, 0.0)
                    signs.add(G.lib.or_phi(G.h, x) > 0.0)
            assert l >= p.amr_uniform
            if len(signs) == 2:
                assert l == R, (X, Y, l)
    for m in maps:
        # 2:1 across faces and corners
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                a = m[max(0, dy):ny + min(0, dy), max(0, dx):nx + min(0, dx)]
                b = m[max(0, -dy):ny + min(0, -dy), max(0, -dx):nx + min(0, -dx)]
                assert np.abs(a.astype(int) - b.astype(int)).max() <= 1
    # Algorithm 1: each coarser grid lowers the highest level by one, its
    # leaves cover the finer ones (nested), and the coarsest is the root grid
    for c, f in zip(maps[:-1], maps[1:]):
        assert c.max() == f.max() - 1
        assert (c <= f).all()
        assert ((f < f.max()) <= (c == f)).all() or (c >= f - 1).all()
    assert (maps[0] == 0).all()
    assert fine.max() == R and fine.min() == p.amr_uniform


def test_hanging_nodes(amr):
    p, lv = amr
    F = lv[-1]
    m = F.leaf_levels()
    ny, nx = m.shape
    R = p.nlevels - 1
    v, par = F.hanging()
    assert len(v) > 0
    free = set(F.free_vertices().tolist())
    for k in range(len(v)):
        X, Y = v[k] % (nx + 1), v[k] // (nx + 1)
        (ax, ay), (bx, by) = [(q % (nx + 1), q // (nx + 1)) for q in par[k]]
        # the midpoint of its parents' edge, parents are free nodes
        assert (ax + bx) == 2 * X and (ay + by) == 2 * Y
        assert par[k][0] in free and par[k][1] in free and v[k] not in free
        # the edge belongs to a leaf one level coarser than the leaves at the node
        s = max(abs(bx - ax), abs(by - ay))
        cells = [(X - 1, Y - 1), (X, Y - 1), (X - 1, Y), (X, Y)]
        lvls = [m[y, x] for x, y in cells if 0 <= x < nx and 0 <= y < ny]
        assert (1 << (R - min(lvls))) == s and max(lvls) == min(lvls) + 1


def _coords(level, nx):
    v = level.free_vertices()
    return v % (nx + 1), v // (nx + 1)


def test_prolongation_exact_on_linear_fields(amr):
    p, lv = amr
    nx = p.n[0]
    for l in range(1, len(lv)):
        F, Cc = lv[l], lv[l - 1]
        Xf, Yf = _coords(F, nx)
        Xc, Yc = _coords(Cc, nx)
        for a, b, c in ((1.0, 0.0, 0.0), (0.3, 1.7, -0.4), (-2.0, 0.5, 3.0)):
            ec = np.zeros(Cc.ndof)
            for k in range(3):
                ec[k::3] = a + b * Xc + c * Yc + k
            got = O.prolong_add(F, Cc, ec, np.zeros(F.ndof))
            _, _, fixed = F.csr()
            for k in range(3):
                want = (a + b * Xf + c * Yf + k) * (~fixed[k::3])
                assert np.abs(got[k::3] - want).max() <= 1e-12 * (1 + np.abs(want).max())


def test_restriction_is_the_transpose():
    p = dataclasses.replace(channel(), alpha=1e-8)
    p.preset = 2
    lv = O.amr_levels(p)
    F, Cc = lv[-1], lv[-2]
    x = inputs.uniform_array(Cc.ndof, 1)
    y = inputs.uniform_array(F.ndof, 2)
    Px = O.prolong_add(F, Cc, x, np.zeros(F.ndof))
    Ry = O.restrict(F, Cc, y)
    assert abs(y @ Px - Ry @ x) <= 1e-12 * abs(y @ Px)


def _interpolate(level, vals, R):
    """The conforming finite element function of free-node values `vals`
    (one component) at every lattice vertex: bilinear on each leaf, hanging
    corners the mean of their parents."""
    m = level.leaf_levels()
    ny, nx = m.shape
    node_of = {int(v): i for i, v in enumerate(level.free_vertices())}
    hv, par = level.hanging()
    hang = {int(v): (int(a), int(b)) for v, (a, b) in zip(hv, par)}

    def corner(v):
        if v in node_of:
            return vals[node_of[v]]
        a, b = hang[v]
        return 0.5 * (vals[node_of[a]] + vals[node_of[b]])
    out = np.zeros((ny + 1) * (nx + 1))
    for Y in range(ny + 1):
        for X in range(nx + 1):
            cx, cy = min(X, nx - 1), min(Y, ny - 1)
            s = 1 << (R - m[cy, cx])
            X0, Y0 = cx // s * s, cy // s * s
            tx, ty = (X - X0) / s, (Y - Y0) / s
            c = [corner((Y0 + (a >> 1) * s) * (nx + 1) + X0 + (a & 1) * s) for a in range(4)]
            out[Y * (nx + 1) + X] = ((1 - tx) * (1 - ty) * c[0] + tx * (1 - ty) * c[1]
                                     + (1 - tx) * ty * c[2] + tx * ty * c[3])
    return out


def test_forms_equal_the_uniform_finest_grid():
    """The conforming adaptive space is a subspace of the uniform finest grid's
    Q1 space.  With alpha = 1 and every boundary point in a finest leaf, the
    velocity and divergence forms of two adaptive functions equal those of
    their interpolants on the uniform finest grid (the Gauss rule is exact on
    the uncut leaves); the pressure stabilisation (a projection on each cell)
    is not refinement-invariant and is left out."""
    p = dataclasses.replace(channel(n=32, nlevels=3, u=0, alpha=1.0), preset=2)
    lv = O.amr_levels(p)
    F = lv[-1]
    R = p.nlevels - 1
    U = O.Level.from_problem(dataclasses.replace(p, amr_uniform=-1))
    bx, _, _, bcell = U.bpoints()
    m = F.leaf_levels()
    nx = p.n[0]
    for c in np.unique(bcell):
        assert m[c // nx, c % nx] == R
    A, _, _ = F.csr()
    Au, _, _ = U.csr()
    nf = F.nnodes
    for seed in range(3):
        u = inputs.uniform_array(F.ndof, 10 + seed)
        v = inputs.uniform_array(F.ndof, 20 + seed)
        ui = np.zeros(U.ndof); vi = np.zeros(U.ndof)
        for k in range(3):
            ui[k::3] = _interpolate(F, u[k::3], R)
            vi[k::3] = _interpolate(F, v[k::3], R)
        for mask_u, mask_v in (((0, 1), (0, 1)), ((0, 1), (2,)), ((2,), (0, 1))):
            uu = np.zeros(F.ndof); vv = np.zeros(F.ndof)
            uf = np.zeros(U.ndof); vf = np.zeros(U.ndof)
            for k in mask_u:
                uu[k::3] = u[k::3]; uf[k::3] = ui[k::3]
            for k in mask_v:
                vv[k::3] = v[k::3]; vf[k::3] = vi[k::3]
            a, b = vv @ (A @ uu), vf @ (Au @ uf)
            assert abs(a - b) <= 1e-11 * (abs(b) + np.abs(A).max()), (seed, mask_u, mask_v, a, b)
    assert nf < U.nnodes


def test_owner_count_is_one(amr):
    p, lv = amr
    for L in lv[1:]:
        cnt = np.zeros(L.ndof, dtype=int)
        _, _, fixed = L.csr()
        for i in range(L.nnodes):
            d, own = L.patch_dofs(i)
            for c in range(3):
                if own[c] >= 0:
                    assert d[own[c]] == i * 3 + c
                    cnt[i * 3 + c] += 1
        assert (cnt[~fixed] == 1).all() and (cnt[fixed] == 0).all()


def test_fgmres_reaches_direct_solution(amr):
    p, lv = amr
    mg = O.MG(p, levels=lv)
    A, b, _ = mg.fine.csr()
    x, its, rel, _ = mg.fgmres(b, rtol=1e-10)
    assert rel <= 1e-10
    xd = spl.spsolve(A.tocsc(), b)
    assert np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)


def test_iteration_counts_bounded_under_refinement():
    """Adding adaptive levels (finer leaves at the circle, fixed 8^2 root and
    uniform level 1) keeps the FGMRES count bounded (Sec. 4)."""
    its = []
    for n, nl in ((32, 3), (64, 4), (128, 5), (256, 6)):
        mg = O.AMRMG(channel(n=n, nlevels=nl, u=1))
        _, k, rel, _ = mg.fgmres(mg.rhs(), rtol=1e-8)
        assert rel <= 1e-8
        its.append(k)
    assert max(its) <= 2 * min(its) + 4, its
