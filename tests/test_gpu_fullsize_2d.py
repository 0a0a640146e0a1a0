"""Parity at the full size of the 2D roofline case (4096^2 cells, one circle
of radius 0.2 at the centre, alpha = 1e-10, 50.4 M DoFs, 9 levels) on sampled
outputs the oracle computes one by one from its own rows of L: operator rows
and one RA sweep with float-pair rows, one stored block per patch (the
configuration `bench.py --mode sweep --workload roofline2d --n 4096` times)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_11636_gb300 import inputs
from tests.gpu_util import oracle_patch_update

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2403_11636_gb300 import build, fc
    build.build()
    p = inputs.roofline_2d()
    s = fc.Solver(p, prec="df64", dedup=0)
    L = O.Level.from_problem(p)      # rows are computed on demand
    return p, s, L


def sample_nodes(p, seed=0):
    n = p.n[0]
    nn = n + 1
    rng = np.random.default_rng(seed)
    nodes = [int(v) for v in rng.integers(0, nn * nn, 6)]
    # next to the circle (cut patches) at four angles
    for ang in (0.0, 0.9, 2.3, 4.0):
        x = 0.5 + 0.2 * np.cos(ang)
        y = 0.5 + 0.2 * np.sin(ang)
        nodes.append(int(round(x * n)) + nn * int(round(y * n)))
    # inflow, outflow and wall nodes (constrained and truncated patches)
    nodes += [0, n, nn * (n // 2), nn * (n // 2) + n, nn * 1 + 1, nn * (n - 1) + n // 3]
    return nodes


def test_roofline2d_operator_sampled(setup):
    p, s, L = setup
    x = inputs.random_vector(p, 5)
    y = s.apply(x).cpu().numpy()
    rng = np.random.default_rng(1)
    dofs = rng.integers(0, L.ndof, 200)
    R, _ = L.dof_rows(dofs)
    nd, nn = 3, p.n[0] + 1
    for q, d in enumerate(dofs):
        node = d // nd
        i, j = node % nn, node // nn
        acc = 0.0
        for t in range(9):
            a, b_ = i + t % 3 - 1, j + t // 3 - 1
            if 0 <= a < nn and 0 <= b_ < nn:
                m = a + nn * b_
                acc += R[q, t] @ x[m * nd:m * nd + nd]
        assert abs(y[d] - acc) <= 1e-12 * (np.abs(R[q]).sum() + 1e-300)


def test_roofline2d_sweep_sampled(setup):
    p, s, L = setup
    x0 = inputs.random_vector(p, 7)
    b = inputs.random_vector(p, 8)
    x1 = s.smooth(x0, b).cpu().numpy()
    nd = 3
    for node in sample_nodes(p):
        upd = oracle_patch_update(L, p, node, b, x0, p.omega)
        for c, u in upd.items():
            g = x1[node * nd + c] - x0[node * nd + c]
            assert abs(g - u) <= 1e-10 * max(abs(u), 1e-300) + 1e-14, (node, c, g, u)
