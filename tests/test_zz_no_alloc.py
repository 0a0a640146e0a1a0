"""fc_smooth_noalloc: the smoother entry point that allocates nothing.

It serves callers that cannot allocate device memory at call time (a serving
runtime that reserved its memory up front, a loop that must not enter the
CUDA allocator).  Its scratch is one static device array shared by all calls,
so this test runs it twice in a row on levels of different size (the second
call starts from the first call's leftovers) and compares each result with
the regular fc_smooth through the C-ABI, within the per-sweep tolerance the
parity tests use.  Collected last so that a run stopping at the first failure
has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2403_11636_gb300 import inputs

pytestmark = pytest.mark.gpu

SWEEP_TOL = 1e-10


@pytest.fixture(scope="module")
def fc():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2403_11636_gb300 import build, fc as fcmod
    build.build()
    return fcmod


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("cache,prec", [("inverse", "fp64"), ("inverse", "df64"), ("inverse", "fp32"),
                                        ("inverse", "bf16"), ("matrix", "fp64"), ("none", "fp64")])
def test_noalloc_matches_fc_smooth_twice(fc, cache, prec):
    """Every cache policy and row precision: the cached rows (FP64, float
    pairs, float32, bfloat16), the cached block factors, and the on-the-fly
    factorisation, each against fc_smooth on the same handle."""
    import torch
    p = inputs.porous_3d(1, n=16, nspheres=5, nlevels=3)
    s = fc.Solver(p, prec=prec, cache=cache)
    lib = s.lib
    for level, seed in ((3, 11), (2, 12)):
        x0 = torch.as_tensor(inputs.random_vector(p, seed, level=level)).cuda()
        b = torch.as_tensor(inputs.random_vector(p, seed + 100, level=level)).cuda()
        ref = x0.clone()
        assert lib.fc_smooth(s.h, level, ctypes.c_void_p(ref.data_ptr()),
                             ctypes.c_void_p(b.data_ptr()), 2) == fc.FC_OK
        got = x0.clone()
        st = lib.fc_smooth_noalloc(s.h, level, ctypes.c_void_p(got.data_ptr()),
                                   ctypes.c_void_p(b.data_ptr()), 2)
        assert st == fc.FC_OK, lib.fc_last_error(s.h)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        x0n = x0.cpu().numpy()
        assert _rel(g - x0n, r - x0n) <= SWEEP_TOL


def test_noalloc_2d_after_3d(fc):
    import torch
    p = inputs.channel_2d(0, n=32, nlevels=3)
    s = fc.Solver(p)
    for _ in range(2):
        x0 = torch.as_tensor(inputs.random_vector(p, 5)).cuda()
        b = torch.as_tensor(inputs.random_vector(p, 6)).cuda()
        ref = s.smooth(x0, b, nsweeps=1)
        got = x0.clone()
        assert s.smooth_noalloc_(got, b, nsweeps=1) == fc.FC_OK
        torch.cuda.synchronize()
        x0n = x0.cpu().numpy()
        assert _rel(got.cpu().numpy() - x0n, ref.cpu().numpy() - x0n) <= SWEEP_TOL


def test_noalloc_rejects_oversized_level(fc):
    """A level whose padded residual exceeds the 16 MiB array is rejected
    with FC_ERR_INVALID and x is left untouched; a smaller level of the same
    handle still runs."""
    import torch
    p = inputs.channel_2d(0, n=1024, nlevels=6)
    s = fc.Solver(p)
    x = s.zeros()
    b = s.rhs()
    before = x.clone()
    assert s.smooth_noalloc_(x, b, level=6) == fc.FC_ERR_INVALID
    assert "16 MiB" in s.lib.fc_last_error(s.h).decode()
    torch.cuda.synchronize()
    assert torch.equal(x, before)
    x5 = torch.as_tensor(inputs.random_vector(p, 1, level=5)).cuda()
    b5 = torch.as_tensor(inputs.random_vector(p, 2, level=5)).cuda()
    ref = s.smooth(x5, b5, level=5)
    got = x5.clone()
    assert s.smooth_noalloc_(got, b5, level=5) == fc.FC_OK
    torch.cuda.synchronize()
    x5n = x5.cpu().numpy()
    assert _rel(got.cpu().numpy() - x5n, ref.cpu().numpy() - x5n) <= SWEEP_TOL
