"""Pins of the adaptive-grid oracle in 3D (oracle/fc_oracle_amr.c on
octrees): cells refined towards a sphere with 2:1 balance across faces,
edges and corners, hanging edge midpoints (two parents) and face centres
(four parents) removed as constraints, and the hierarchy of Algorithm 1
(Sec. 3).

The pins are those of the 2D quadtree pins, restated for octrees: a tree
refined uniformly is the uniform 3D grid (operator, load, Dirichlet data
including the product inflow profile, patches, trilinear prolongation); the
refinement, balance and coarsening rules checked cell by cell on the level
map; the hanging-node geometry; exactness of the prolongation on linear
fields; the adaptive bilinear forms equal those of the uniform finest grid
on the interpolated functions (the adaptive space is a conforming subspace);
one owner per free DoF; FGMRES reaching the direct solution."""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

from oracle import oracle as O
from paper_2403_11636_gb300 import inputs


def box3(n=16, nlevels=3, u=1, alpha=1e-8, preset=0, r=0.2, c=(0.45, 0.5, 0.55)):
    """Unit cube with one sphere; lattice n^3 (the finest cells)."""
    shapes = np.array([[0.0, c[0], c[1], c[2], r, r, r, 1.0, 0.0]])
    return inputs.Problem(name=f"box3_n{n}", dim=3, n=(n, n, n), lo=(0.0,) * 3, hi=(1.0,) * 3, shapes=shapes,
                          alpha=alpha, qdepth=2, nlevels=nlevels, preset=preset, force_kind=0,
                          force=(1.0, 0.5, -0.25), amr_uniform=u)


@pytest.fixture(scope="module")
def amr3():
    """Leaves of levels 0 to 2 (root 4^3, lattice 16^3), so that the 2:1
    balance has work to do."""
    p = box3(u=0)
    return p, O.amr_levels(p)


def _xyz(v, n):
    return v % (n + 1), (v // (n + 1)) % (n + 1), v // ((n + 1) * (n + 1))


def test_uniform_octree_is_the_uniform_grid():
    p = box3(n=8, nlevels=3, u=2)
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
            d1, o1 = U.patch_dofs(node)
            d2, o2 = lv[l - 1].patch_dofs(node)
            assert np.array_equal(d1, d2) and np.array_equal(o1, o2)
    # the inflow data is the product of the two parabolas
    A, b, fixed = lv[-1].csr()
    x, y, z = _xyz(lv[-1].free_vertices(), p.n[0])
    inflow = (x == 0) & (y > 0) & (y < p.n[1]) & (z > 0) & (z < p.n[2])
    sy, sz = y / p.n[1], z / p.n[2]
    want = 4.0 * p.ubar * sy * (1 - sy) * 4.0 * sz * (1 - sz)
    assert fixed[0::4][inflow].all() and np.abs(b[0::4][inflow] - want[inflow]).max() <= 1e-15
    # prolongation equals the uniform trilinear interpolation
    F, Cc = lv[2], lv[1]
    UF, UC = O.Level.from_problem(p, 3), O.Level.from_problem(p, 2)
    UF.assemble(); UC.assemble()
    e = inputs.uniform_array(Cc.ndof, 5)
    xf = inputs.uniform_array(F.ndof, 6)
    assert np.abs(O.prolong_add(F, Cc, e, xf) - O.prolong_add(UF, UC, e, xf)).max() <= 1e-15


def test_octree_refinement_balance_and_algorithm_1(amr3):
    p, lv = amr3
    R = p.nlevels - 1
    maps = [l.leaf_levels() for l in lv]
    fine = maps[-1]
    G = O.Level.from_problem(p)
    nz, ny, nx = fine.shape
    h = [(p.hi[k] - p.lo[k]) / p.n[k] for k in range(3)]
    ncut = 0
    for Z in range(nz):
        for Y in range(ny):
            for X in range(nx):
                l = fine[Z, Y, X]
                s = 1 << (R - l)
                if X % s or Y % s or Z % s:
                    continue
                signs = set()
                for k in range(3):
                    for j in range(3):
                        for i in range(3):
                            pt = (O.C.c_double * 3)(p.lo[0] + (X + 0.5 * i * s) * h[0],
                                                    p.lo[1] + (Y + 0.5 * j * s) * h[1],
                                                    p.lo[2] + (Z + 0.5 * k * s) * h[2])
                            signs.add(G.lib.or_phi(G.h, pt) > 0.0)
                assert l >= p.amr_uniform
                if len(signs) == 2:
                    assert l == R, (X, Y, Z, l)
                    ncut += 1
    assert ncut > 0
    for m in maps:
        # 2:1 across faces, edges and corners (all 26 neighbours)
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    a = m[max(0, dz):nz + min(0, dz), max(0, dy):ny + min(0, dy), max(0, dx):nx + min(0, dx)]
                    b = m[max(0, -dz):nz + min(0, -dz), max(0, -dy):ny + min(0, -dy), max(0, -dx):nx + min(0, -dx)]
                    assert np.abs(a.astype(int) - b.astype(int)).max() <= 1
        # leaves are aligned cubes of their level
        for Z in range(nz):
            for Y in range(ny):
                for X in range(nx):
                    s = 1 << (R - m[Z, Y, X])
                    Z0, Y0, X0 = Z // s * s, Y // s * s, X // s * s
                    assert (m[Z0:Z0 + s, Y0:Y0 + s, X0:X0 + s] == m[Z, Y, X]).all()
    # Algorithm 1: each coarser grid lowers the highest level by one, its
    # leaves cover the finer ones, and the coarsest is the root grid
    for c, f in zip(maps[:-1], maps[1:]):
        assert c.max() == f.max() - 1
        assert (c <= f).all() and (c >= f - 1).all()
        assert (c[f == f.max()] == f.max() - 1).all()
    assert (maps[0] == 0).all()
    assert fine.max() == R and fine.min() == p.amr_uniform


def test_octree_hanging_nodes(amr3):
    p, lv = amr3
    F = lv[-1]
    m = F.leaf_levels()
    n = p.n[0]
    R = p.nlevels - 1
    v, par = F.hanging()
    free = set(F.free_vertices().tolist())
    kinds = {2: 0, 4: 0}
    for k in range(len(v)):
        X, Y, Z = _xyz(v[k], n)
        ps = [q for q in par[k] if q >= 0]
        kinds[len(ps)] += 1
        P = np.array([_xyz(q, n) for q in ps])
        # the centre of its parents, which are free nodes
        assert (P.sum(axis=0) == len(ps) * np.array([X, Y, Z])).all()
        assert all(q in free for q in ps) and v[k] not in free
        ext = P.max(axis=0) - P.min(axis=0)
        s = ext.max()
        if len(ps) == 2:   # an edge of length s along one axis
            assert sorted(ext.tolist()) == [0, 0, s]
        else:              # a face: a square of side s normal to one axis
            assert sorted(ext.tolist()) == [0, s, s]
            assert len({tuple(q) for q in P}) == 4
        # leaves at the node: the coarse one with that edge or face, and finer ones
        lvls = [m[z, y, x] for z in (Z - 1, Z) for y in (Y - 1, Y) for x in (X - 1, X)
                if 0 <= x < n and 0 <= y < n and 0 <= z < n]
        assert (1 << (R - min(lvls))) == s and max(lvls) == min(lvls) + 1
    assert kinds[2] > 0 and kinds[4] > 0


def test_octree_prolongation_exact_on_linear_fields(amr3):
    p, lv = amr3
    n = p.n[0]
    for l in range(1, len(lv)):
        F, Cc = lv[l], lv[l - 1]
        Xf, Yf, Zf = _xyz(F.free_vertices(), n)
        Xc, Yc, Zc = _xyz(Cc.free_vertices(), n)
        _, _, fixed = F.csr()
        for a, b, c, d in ((1.0, 0.0, 0.0, 0.0), (0.3, 1.7, -0.4, 0.9), (-2.0, 0.5, 3.0, -1.1)):
            ec = np.zeros(Cc.ndof)
            for k in range(4):
                ec[k::4] = a + b * Xc + c * Yc + d * Zc + k
            got = O.prolong_add(F, Cc, ec, np.zeros(F.ndof))
            for k in range(4):
                want = (a + b * Xf + c * Yf + d * Zf + k) * (~fixed[k::4])
                assert np.abs(got[k::4] - want).max() <= 1e-12 * (1 + np.abs(want).max())


def test_octree_restriction_is_the_transpose():
    p = box3(preset=2)
    lv = O.amr_levels(p)
    F, Cc = lv[-1], lv[-2]
    x = inputs.uniform_array(Cc.ndof, 1)
    y = inputs.uniform_array(F.ndof, 2)
    Px = O.prolong_add(F, Cc, x, np.zeros(F.ndof))
    Ry = O.restrict(F, Cc, y)
    assert abs(y @ Px - Ry @ x) <= 1e-12 * abs(y @ Px)


def _interpolate3(level, vals, n, R):
    """The conforming finite element function of free-node values `vals`
    (one component) at every lattice vertex: trilinear on each leaf, a
    hanging corner the mean of its parents."""
    m = level.leaf_levels()
    node_of = {int(v): i for i, v in enumerate(level.free_vertices())}
    hv, par = level.hanging()
    hang = {int(v): [int(q) for q in pp if q >= 0] for v, pp in zip(hv, par)}

    def corner(v):
        if v in node_of:
            return vals[node_of[v]]
        ps = hang[v]
        return sum(vals[node_of[q]] for q in ps) / len(ps)
    n1 = n + 1
    out = np.zeros(n1 ** 3)
    for Z in range(n1):
        for Y in range(n1):
            for X in range(n1):
                cx, cy, cz = min(X, n - 1), min(Y, n - 1), min(Z, n - 1)
                s = 1 << (R - m[cz, cy, cx])
                X0, Y0, Z0 = cx // s * s, cy // s * s, cz // s * s
                t = ((X - X0) / s, (Y - Y0) / s, (Z - Z0) / s)
                acc = 0.0
                for a in range(8):
                    w = 1.0
                    for k in range(3):
                        w *= t[k] if (a >> k) & 1 else 1.0 - t[k]
                    if w == 0.0:
                        continue
                    vtx = ((Z0 + ((a >> 2) & 1) * s) * n1 + Y0 + ((a >> 1) & 1) * s) * n1 + X0 + (a & 1) * s
                    acc += w * corner(vtx)
                out[(Z * n1 + Y) * n1 + X] = acc
    return out


def test_octree_forms_equal_the_uniform_finest_grid():
    """With alpha = 1 and every boundary point in a finest leaf, the velocity
    and divergence forms of two adaptive functions equal those of their
    interpolants on the uniform finest grid (the Gauss rule is exact on the
    uncut leaves); the pressure stabilisation (a projection on each cell) is
    not refinement-invariant and is left out."""
    p = box3(n=16, nlevels=3, u=0, alpha=1.0, preset=2)
    lv = O.amr_levels(p)
    F = lv[-1]
    R = p.nlevels - 1
    n = p.n[0]
    U = O.Level.from_problem(p)
    _, _, _, bcell = U.bpoints()
    m = F.leaf_levels()
    for c in np.unique(bcell):
        assert m[c // (n * n), (c // n) % n, c % n] == R
    assert (m < R).any()
    A, _, _ = F.csr()
    Au, _, _ = U.csr()
    for seed in range(2):
        u = inputs.uniform_array(F.ndof, 10 + seed)
        v = inputs.uniform_array(F.ndof, 20 + seed)
        ui = np.zeros(U.ndof); vi = np.zeros(U.ndof)
        for k in range(4):
            ui[k::4] = _interpolate3(F, u[k::4], n, R)
            vi[k::4] = _interpolate3(F, v[k::4], n, R)
        for mask_u, mask_v in (((0, 1, 2), (0, 1, 2)), ((0, 1, 2), (3,)), ((3,), (0, 1, 2))):
            uu = np.zeros(F.ndof); vv = np.zeros(F.ndof)
            uf = np.zeros(U.ndof); vf = np.zeros(U.ndof)
            for k in mask_u:
                uu[k::4] = u[k::4]; uf[k::4] = ui[k::4]
            for k in mask_v:
                vv[k::4] = v[k::4]; vf[k::4] = vi[k::4]
            a, b = vv @ (A @ uu), vf @ (Au @ uf)
            assert abs(a - b) <= 1e-11 * (abs(b) + np.abs(A).max()), (seed, mask_u, mask_v, a, b)
    assert F.nnodes < U.nnodes


def test_octree_owner_count_is_one(amr3):
    p, lv = amr3
    for L in lv[1:]:
        cnt = np.zeros(L.ndof, dtype=int)
        _, _, fixed = L.csr()
        for i in range(L.nnodes):
            d, own = L.patch_dofs(i)
            for c in range(4):
                if own[c] >= 0:
                    assert d[own[c]] == i * 4 + c
                    cnt[i * 4 + c] += 1
        assert (cnt[~fixed] == 1).all() and (cnt[fixed] == 0).all()


def test_octree_fgmres_reaches_direct_solution():
    """alpha = 1e-4 keeps the fictitious part well enough conditioned for the
    sparse direct solve to serve as the reference at 1e-8."""
    p = box3(alpha=1e-4)
    mg = O.MG(p, levels=O.amr_levels(p))
    A, b, _ = mg.fine.csr()
    x, its, rel, _ = mg.fgmres(b, rtol=1e-10)
    assert rel <= 1e-10
    xd = spl.spsolve(A.tocsc(), b)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
