"""The bad-cut rule for reduced-precision rows (fc_options.badcut_frac).

Float32 / bfloat16 rows come from float32 factors with iterative refinement.
A patch whose smallest cut-cell fluid fraction over the 4^d cells between
its velocity nodes is below badcut_frac (1e-3 by default) takes the
float-pair (FP64-class) factorisation instead: the higher-precision
factorisation of badly cut, ill-conditioned patch blocks (Sec. 3.1.2; the
mixed-precision configuration's 1e-3 cut-volume rule).

The expected set of patches is computed here from the oracle's own cell
fluid volumes and compared with the library's count exactly; the flagged
patches' stored rows must equal the float-pair rows of the same problem
rounded to float32.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_11636_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2403_11636_gb300 import build, fc as fcmod
    build.build()
    return fcmod


def flagged_patches(p, frac):
    """{level: sorted node list} of the patches the rule selects, from the
    oracle's cell fluid volumes (levels 2..L carry patch caches)."""
    out = {}
    for lv in range(2, p.nlevels + 1):
        L = O.Level.from_problem(p, lv)
        n = p.level_n(lv)
        vol = float(np.prod([(p.hi[k] - p.lo[k]) / n[k] for k in range(p.dim)]))
        nodes = set()
        for c in range(L.ncell):
            f = L.cell_element(c)["fluid_volume"] / vol
            if not (0.0 < f < 1.0 and f < frac):
                continue
            cx, cy = c % n[0], c // n[0]
            # patches i with the cell among cells i-2 .. i+1
            for iy in range(cy - 1, cy + 3):
                for ix in range(cx - 1, cx + 3):
                    if 0 <= ix <= n[0] and 0 <= iy <= n[1]:
                        nodes.add(ix + (n[0] + 1) * iy)
        out[lv] = sorted(nodes)
    return out


@pytest.mark.parametrize("seed", [63, 7])
def test_badcut_rule_counts_and_rows(fc, seed):
    p = inputs.batch_2d(seed)
    want = flagged_patches(p, 1e-3)
    total = sum(len(v) for v in want.values())
    assert total > 0
    s32 = fc.Solver(p, prec="fp32", badcut_frac=1e-3)
    assert s32.info()["bytes"][7] == total
    off = fc.Solver(p, prec="fp32", badcut_frac=0.0)
    assert off.info()["bytes"][7] == 0
    off.close()
    sdf = fc.Solver(p, prec="df64")
    for node in want[p.nlevels]:
        a = s32.patch_rows(node)
        b = sdf.patch_rows(node)
        # float-pair rows rounded to float32: within half an ulp of float32
        assert np.all(np.abs(a - b) <= 2.0 ** -24 * np.abs(b) * 1.0001 + 1e-300), node
    # the solve still reaches the mixed-precision bar
    _, its, rr = s32.solve(s32.rhs(), rtol=1e-8, maxit=400)
    assert rr <= 1e-8
    s32.close()
    sdf.close()
