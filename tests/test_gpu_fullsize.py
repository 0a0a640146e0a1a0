"""Parity at the full 64^3 porous-medium size (the benchmark workload: 64^3
cells, 40 spheres, 5 levels, 274,625 patches on the finest level) on sampled
outputs the oracle computes one by one from its own rows of L, for every
patch-row precision.  At this size the library takes its large-level kernels
(one thread per node in the float-pair residual, the persistent float-pair
apply over all patches), which the small parity cases never reach.

Per-update bounds (relative to the oracle's update u and to the magnitude
S = omega sum_j |c_j r_j| that the rounding of the patch dot product scales
with):
  fp64  |g - u| <= 1e-10 |u| + 1e-14             (the per-sweep FP64 bound)
  df64  |g - u| <= 1e-10 |u| + 1e-11 S           (rows from the float-pair
                                                  elimination, ~1e-12 of their
                                                  scale, and 402 pair products
                                                  within 2^-48 relative each)
  fp32  |g - u| <= 3e-5 S                        (402 float32 FMAs on rows and
                                                  residual rounded to float32)
  bf16  |g - u| <= 5e-3 S                        (rows rounded to bfloat16,
                                                  2^-8 relative, + the float32
                                                  sum)
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_11636_gb300 import inputs
from tests.gpu_util import oracle_patch_update, rel

pytestmark = pytest.mark.gpu

PRECS = ["fp64", "df64", "fp32", "bf16"]


@pytest.fixture(scope="module")
def base():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2403_11636_gb300 import build, fc
    build.build()
    p = inputs.porous_3d(0)          # 64^3, 40 spheres, 5 levels
    L = O.Level.from_problem(p)      # not assembled: rows are computed on demand
    return p, L, fc, {}


def solver(base, prec):
    p, _, fc, cache = base
    if prec not in cache:
        cache[prec] = fc.Solver(p, prec=prec, dedup=0)
    return cache[prec]


def sample_nodes(p, k=4, seed=0):
    n = p.n[0]
    nn = n + 1
    rng = np.random.default_rng(seed)
    nodes = list(rng.integers(0, nn ** 3, k))
    # nodes next to sphere surfaces (cut patches)
    for sh in p.shapes[:k]:
        c, r = sh[1:4], sh[4]
        pt = c + r * np.array([1.0, 0.0, 0.0])
        ijk = np.clip(np.round(pt * n).astype(int), 0, n)
        nodes.append(int(ijk[0] + nn * (ijk[1] + nn * ijk[2])))
    # inside a sphere (fictitious patch)
    c = p.shapes[0][1:4]
    ijk = np.clip(np.round(c * n).astype(int), 0, n)
    nodes.append(int(ijk[0] + nn * (ijk[1] + nn * ijk[2])))
    # boundary nodes (constrained walls, truncated patches)
    nodes += [0, nn - 1, nn * nn * (nn - 1) + 5, 3 + nn * 1 + nn * nn * 7, 1 + nn * 2 + nn * nn * 32]
    return [int(v) for v in nodes]


def test_fullsize_operator_sampled(base):
    p, L, _, _ = base
    s = solver(base, "fp64")
    x = inputs.random_vector(p, 5)
    y = s.apply(x).cpu().numpy()
    rng = np.random.default_rng(1)
    dofs = rng.integers(0, L.ndof, 300)
    R, _ = L.dof_rows(dofs)
    nd, nn = 4, p.n[0] + 1
    for q, d in enumerate(dofs):
        node = d // nd
        i, j, k = node % nn, (node // nn) % nn, node // (nn * nn)
        acc = 0.0
        for t in range(27):
            a, b_, c = i + t % 3 - 1, j + (t // 3) % 3 - 1, k + t // 9 - 1
            if 0 <= a < nn and 0 <= b_ < nn and 0 <= c < nn:
                acc += R[q, t] @ x[(a + nn * (b_ + nn * c)) * nd:(a + nn * (b_ + nn * c)) * nd + nd]
        assert abs(y[d] - acc) <= 1e-12 * (np.abs(R[q]).sum() + 1e-300)


def _bound(prec, u, scale):
    if prec == "fp64":
        return 1e-10 * abs(u) + 1e-14
    if prec == "df64":
        return 1e-10 * abs(u) + 1e-11 * scale
    if prec == "fp32":
        return 3e-5 * scale
    return 5e-3 * scale


@pytest.mark.parametrize("prec", PRECS)
def test_fullsize_sweep_sampled(base, prec):
    """One sweep of the finest level through fc_smooth with each row
    precision: sampled owned-DoF updates (interior, cut, fictitious, wall and
    truncated patches) against the oracle's rows of L and L_i^{-1}."""
    p, L, _, _ = base
    s = solver(base, prec)
    x0 = inputs.random_vector(p, 7)
    b = inputs.random_vector(p, 8)
    x1 = s.smooth(x0, b).cpu().numpy()
    nd = 4
    checked = 0
    for node in sample_nodes(p):
        upd, scale = oracle_patch_update(L, p, node, b, x0, p.omega, with_scale=True)
        for c, u in upd.items():
            g = x1[node * nd + c] - x0[node * nd + c]
            assert abs(g - u) <= _bound(prec, u, scale[c]), (prec, node, c, g, u, scale[c])
            checked += 1
    assert checked >= 40


def test_fullsize_vcycle_pairs_match_fp64(base):
    """The timed float-pair V-cycle (pair residual and persistent pair apply
    on the 64^3 level, FP64 transfers and coarse solve) agrees with the FP64
    V-cycle to the per-sweep bound; the FP64 V-cycle itself matches the
    oracle's at the sizes the oracle finishes (test_gpu_parity,
    test_gpu_midsize)."""
    p, _, _, _ = base
    s64, sdf = solver(base, "fp64"), solver(base, "df64")
    x0 = inputs.random_vector(p, 71)
    b = inputs.random_vector(p, 72)
    v64 = s64.vcycle(x0, b).cpu().numpy()
    vdf = sdf.vcycle(x0, b).cpu().numpy()
    assert rel(vdf - x0, v64 - x0) <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_fullsize_fgmres(base, prec):
    """Full 64^3 solve to 1e-8: the library's true residual, the oracle's own
    rows of L applied to the GPU solution at sampled DoFs, and the same
    iteration count for FP64 and float-pair rows."""
    p, L, _, cache = base
    s = solver(base, prec)
    b = s.rhs()
    x, its, rr = s.solve(b, rtol=1e-8, maxit=200)
    assert rr <= 1e-8 and its <= 60
    cache.setdefault("its", {})[prec] = its
    xb = x.cpu().numpy()
    bb = b.cpu().numpy()
    rng = np.random.default_rng(2)
    dofs = rng.integers(0, L.ndof, 200)
    R, rhs = L.dof_rows(dofs)
    np.testing.assert_allclose(rhs, bb[dofs], rtol=1e-11, atol=1e-20)
    nd, nn = 4, p.n[0] + 1
    res = []
    for q, d in enumerate(dofs):
        node = d // nd
        i, j, k = node % nn, (node // nn) % nn, node // (nn * nn)
        acc = 0.0
        for t in range(27):
            a, b_, c = i + t % 3 - 1, j + (t // 3) % 3 - 1, k + t // 9 - 1
            if 0 <= a < nn and 0 <= b_ < nn and 0 <= c < nn:
                m = a + nn * (b_ + nn * c)
                acc += R[q, t] @ xb[m * nd:m * nd + nd]
        res.append(rhs[q] - acc)
    # the sampled residual is part of the full one (<= 1e-8 ||b||); 1e-7
    # leaves room for the rounding of the oracle's own row products
    assert np.linalg.norm(res) <= 1e-7 * np.linalg.norm(bb)
    if len(cache["its"]) == 2:
        assert cache["its"]["fp64"] == cache["its"]["df64"], cache["its"]
