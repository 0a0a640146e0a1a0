"""The binding's vector checks, without a GPU.

Every call of the C-ABI that takes a vector reads or writes exactly the
level's DoF count of float64 values at the pointer it is given, so the
binding rejects anything else before the pointer leaves Python.  A CUDA
tensor is stood in for by an object with the same attributes (there is no
GPU here); the torch module is passed in, so the stand-in is accepted
exactly where a real tensor would be.
"""
import types

import numpy as np
import pytest
import torch

from paper_2403_11636_gb300 import fc


class FakeCudaTensor:
    def __init__(self, n, dtype=torch.float64, contiguous=True, index=0):
        self.shape = (n,)
        self.dtype = dtype
        self.device = types.SimpleNamespace(index=index, type="cuda")
        self.is_cuda = True
        self._n, self._c = n, contiguous

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._c


FAKE_TORCH = types.SimpleNamespace(is_tensor=lambda t: isinstance(t, (torch.Tensor, FakeCudaTensor)),
                                   float64=torch.float64)


def rejects(fn, *args, **kw):
    with pytest.raises(fc.FcError) as e:
        fn(*args, **kw)
    assert e.value.code == fc.FC_ERR_INVALID
    return str(e.value)


def test_device_vector_accepted():
    t = FakeCudaTensor(12)
    assert fc.check_device_vector(FAKE_TORCH, t, 12, 0, "x") is t


@pytest.mark.parametrize("bad", [
    FakeCudaTensor(11),                            # wrong length
    FakeCudaTensor(12, dtype=torch.float32),       # wrong type
    FakeCudaTensor(12, contiguous=False),          # strided view
    FakeCudaTensor(12, index=1),                   # another GPU
    torch.zeros(12, dtype=torch.float64),          # host memory
    np.zeros(12),                                  # not a tensor
], ids=["length", "dtype", "strided", "device", "host tensor", "numpy"])
def test_device_vector_rejected(bad):
    msg = rejects(fc.check_device_vector, FAKE_TORCH, bad, 12, 0, "x")
    assert "x: expected a contiguous float64 tensor of 12 values on cuda:0" in msg


def test_host_vector_checks():
    a = np.zeros(10)
    assert fc.check_host_vector(torch, a, 10, "b_host") is a
    t = torch.zeros(10, dtype=torch.float64)
    assert fc.check_host_vector(torch, t, 10, "x_host", writable=True) is t
    rejects(fc.check_host_vector, torch, np.zeros(9), 10, "b_host")
    rejects(fc.check_host_vector, torch, np.zeros(10, dtype=np.float32), 10, "b_host")
    rejects(fc.check_host_vector, torch, np.zeros(20)[::2], 10, "b_host")
    rejects(fc.check_host_vector, torch, torch.zeros(10, dtype=torch.float32), 10, "b_host")
    rejects(fc.check_host_vector, torch, [0.0] * 10, 10, "b_host")
    ro = np.zeros(10)
    ro.setflags(write=False)
    assert fc.check_host_vector(torch, ro, 10, "b_host") is ro
    rejects(fc.check_host_vector, torch, ro, 10, "x_host", writable=True)


def test_solver_needs_a_gpu():
    """Without a GPU the binding refuses to set anything up (no CPU path)."""
    from paper_2403_11636_gb300 import inputs
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rejects_any = pytest.raises(fc.FcError)
    with rejects_any:
        fc.Solver(inputs.channel_2d(0, n=8, nlevels=1))


def test_batch_refuses_to_run_on_closed_solvers():
    """A batch works on its solvers' device data; once one of them (or the
    batch) is closed, every batch call is refused before it reaches the
    library.  The batch object is assembled by hand here (no GPU)."""
    import ctypes as C
    B = object.__new__(fc.Batch)
    B.torch = torch
    B.b = C.c_void_p(0x1000)          # stands for an open batch; never passed on
    B.solvers = [types.SimpleNamespace(h=C.c_void_p(0x2000)), types.SimpleNamespace(h=C.c_void_p())]
    B.offsets, B.device = [0, 4, 8], 0
    x = FakeCudaTensor(8)
    for call in (lambda: B.smooth_(x, x), lambda: B.vcycle_(x, x), lambda: B.solve(x),
                 lambda: B.solve_host(np.zeros(8), np.zeros(8))):
        assert "solver of this batch was closed" in rejects(call)
    B.solvers[1].h = C.c_void_p(0x3000)
    B.b = C.c_void_p()
    assert "batch was closed" in rejects(lambda: B.smooth_(x, x))
