"""The 128^3 porous-medium configuration with 300 spheres (8.6 M DoFs):
mixed-precision patch rows inside the FP64 FGMRES.  The oracle cannot solve
this size, so the check is (i) the library's true FP64 residual, (ii) the
oracle's own rows of L at sampled DoFs applied to the GPU solution, and
(iii) agreement with the float-pair-row solve to 1e-6 in velocity and
pressure."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_11636_gb300 import inputs
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2403_11636_gb300 import build, fc
    build.build()
    p = inputs.porous_3d(0, n=128, nspheres=300, nlevels=6)
    return p, fc


def test_128_mixed_precision_solve(big):
    p, fc = big
    s32 = fc.Solver(p, prec="fp32", dedup=1)
    b = s32.rhs()
    x32, its32, rr32 = s32.solve(b, rtol=1e-8, maxit=300)
    assert rr32 <= 1e-8
    xs = x32.cpu().numpy()
    bs = b.cpu().numpy()
    s32.close()
    del s32
    # oracle rows at sampled DoFs applied to the GPU solution
    L = O.Level.from_problem(p)
    rng = np.random.default_rng(5)
    dofs = rng.integers(0, L.ndof, 200)
    R, rhs = L.dof_rows(dofs)
    np.testing.assert_allclose(rhs, bs[dofs], rtol=1e-10, atol=1e-20)
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
                acc += R[q, t] @ xs[m * nd:m * nd + nd]
        res.append(rhs[q] - acc)
    assert np.linalg.norm(res) <= 1e-6 * np.linalg.norm(bs)
    # float-pair rows: same solution to the tolerance
    sdf = fc.Solver(p, prec="df64", dedup=1)
    xdf, itsdf, rrdf = sdf.solve(sdf.rhs(), rtol=1e-10, maxit=300)
    xd = xdf.cpu().numpy()
    for comp in ([0, 1, 2], [3]):
        idx = np.concatenate([np.arange(c, len(xd), nd) for c in comp])
        assert rel(xs[idx], xd[idx]) <= 1e-6
