"""ctypes binding of libfc (include/fc.h): argument marshalling only.

Every numerical step runs in the CUDA library; this module allocates device
vectors with PyTorch and passes their pointers.  There is no CPU fallback:
importing it on a machine without the built library or without a GPU raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfc.so")

FC_OK, FC_ERR_INVALID, FC_ERR_OOM, FC_ERR_CUDA = 0, 1, 2, 3
FC_ERR_NOT_CONVERGED, FC_ERR_SINGULAR, FC_ERR_TIMEOUT = 4, 5, 6
CACHE = {"inverse": 0, "matrix": 1, "none": 2}
PREC = {"fp64": 0, "fp32": 1, "bf16": 2, "df64": 3}
EXPORTS = ("fc_options_default", "fc_setup", "fc_rhs", "fc_residual", "fc_apply", "fc_smooth",
           "fc_smooth_noalloc", "fc_restrict", "fc_prolong_add", "fc_coarse_solve", "fc_vcycle", "fc_solve",
           "fc_gmg_solve", "fc_solve_host", "fc_info", "fc_patch_rows", "fc_patch_dofs", "fc_footprint_estimate",
           "fc_profile_enable", "fc_profile_read", "fc_launch_count", "fc_probe_fma_rate", "fc_sync", "fc_last_error",
           "fc_destroy", "fc_batch_create", "fc_batch_create_tiled", "fc_batch_offsets", "fc_batch_tile", "fc_batch_set_tile",
           "fc_batch_smooth", "fc_batch_vcycle", "fc_batch_solve", "fc_batch_solve_host", "fc_batch_info", "fc_batch_profile_enable",
           "fc_batch_profile_read", "fc_batch_sync",
           "fc_batch_last_error", "fc_batch_destroy")


class FcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libfc error {code}: {msg}")
        self.code = code


def _describe(t) -> str:
    if hasattr(t, "dtype") and hasattr(t, "shape"):
        dev = getattr(t, "device", "host")
        return f"{type(t).__name__} {tuple(t.shape)} {t.dtype} on {dev}"
    return type(t).__name__


def check_device_vector(torch, t, n: int, device: int, name: str):
    """The library reads or writes exactly n float64 values at a device
    pointer: anything else is rejected here, before the pointer reaches a
    kernel (a host pointer, a short vector or another GPU's memory would be
    an illegal access on the device)."""
    ok = (torch.is_tensor(t) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
          and t.numel() == n and (t.device.index if t.device.index is not None else 0) == device)
    if not ok:
        raise FcError(FC_ERR_INVALID, f"{name}: expected a contiguous float64 tensor of {n} values on "
                                      f"cuda:{device}, got {_describe(t)}")
    return t


def check_host_vector(torch, a, n: int, name: str, writable: bool = False):
    """A host buffer of exactly n contiguous float64 values (numpy array or
    CPU tensor, pinned or not); ``writable`` for a buffer the call fills."""
    if torch.is_tensor(a):
        ok = (not a.is_cuda) and a.dtype == torch.float64 and a.is_contiguous() and a.numel() == n
    else:
        ok = (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
              and a.size == n and (a.flags["WRITEABLE"] or not writable))
    if not ok:
        raise FcError(FC_ERR_INVALID, f"{name}: expected {n} contiguous float64 host values, got {_describe(a)}")
    return a


class FcShape(C.Structure):
    _fields_ = [("type", C.c_int), ("c", C.c_double * 3), ("r", C.c_double * 3),
                ("rot", C.c_double * 2)]


class FcGrid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3)]


class FcLevelset(C.Structure):
    _fields_ = [("nshapes", C.c_int), ("shapes", C.POINTER(FcShape))]


class FcOptions(C.Structure):
    _fields_ = [("eta", C.c_double), ("nitsche_beta", C.c_double), ("omega", C.c_double),
                ("nu_pre", C.c_int), ("nu_post", C.c_int), ("quad_depth", C.c_int),
                ("cache", C.c_int), ("prec", C.c_int), ("fgmres_restart", C.c_int),
                ("bc_preset", C.c_int), ("ubar", C.c_double), ("force_kind", C.c_int),
                ("force", C.c_double * 3), ("dedup", C.c_int), ("tc", C.c_int), ("badcut_frac", C.c_double),
                ("element", C.c_int), ("galerkin", C.c_int), ("amr_uniform", C.c_int)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libfc.so; raises if it is missing (build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FcError(-1, f"{path} not built; run paper_2403_11636_gb300.build.build()")
    lib = C.CDLL(path)
    vp, d, i, ll = C.c_void_p, C.c_double, C.c_int, C.c_longlong
    P = C.POINTER
    lib.fc_options_default.argtypes = [P(FcOptions)]
    lib.fc_setup.argtypes = [P(vp), P(FcGrid), P(FcLevelset), d, i, P(FcOptions), vp]
    lib.fc_rhs.argtypes = [vp, vp]
    lib.fc_residual.argtypes = [vp, i, vp, vp, vp]
    lib.fc_apply.argtypes = [vp, i, vp, vp]
    lib.fc_smooth.argtypes = [vp, i, vp, vp, i]
    lib.fc_smooth_noalloc.argtypes = [vp, i, vp, vp, i]
    lib.fc_restrict.argtypes = [vp, i, vp, vp]
    lib.fc_prolong_add.argtypes = [vp, i, vp, vp]
    lib.fc_coarse_solve.argtypes = [vp, vp, vp]
    lib.fc_vcycle.argtypes = [vp, vp, vp]
    lib.fc_solve.argtypes = [vp, vp, vp, d, i, P(i), P(d)]
    lib.fc_solve_host.argtypes = [vp, vp, vp, d, i, P(i), P(d)]
    lib.fc_gmg_solve.argtypes = [vp, vp, vp, d, i, P(i), P(d)]
    lib.fc_info.argtypes = [vp, i, P(ll), P(ll), P(C.c_size_t)]
    lib.fc_patch_rows.argtypes = [vp, i, ll, P(d)]
    lib.fc_footprint_estimate.restype = C.c_size_t
    lib.fc_footprint_estimate.argtypes = [P(FcGrid), i, P(FcOptions)]
    lib.fc_profile_enable.argtypes = [vp, i]
    lib.fc_profile_read.argtypes = [vp, i, P(ll), P(d), P(d)]
    lib.fc_launch_count.argtypes = [P(ll)]
    lib.fc_probe_fma_rate.argtypes = [i, P(d), P(d)]
    lib.fc_sync.argtypes = [vp]
    lib.fc_last_error.restype = C.c_char_p
    lib.fc_last_error.argtypes = [vp]
    lib.fc_destroy.argtypes = [vp]
    lib.fc_batch_create.argtypes = [P(vp), P(vp), i, vp]
    lib.fc_batch_offsets.argtypes = [vp, P(ll)]
    lib.fc_batch_tile.argtypes = [vp, P(i), P(i), P(i)]
    lib.fc_batch_set_tile.argtypes = [vp, i, i, i]
    lib.fc_batch_create_tiled.argtypes = [P(vp), P(vp), i, vp, i, i, i]
    lib.fc_batch_smooth.argtypes = [vp, vp, vp, i]
    lib.fc_batch_vcycle.argtypes = [vp, vp, vp]
    lib.fc_batch_solve.argtypes = [vp, vp, vp, d, i, P(i), P(d)]
    lib.fc_batch_solve_host.argtypes = [vp, vp, vp, d, i, P(i), P(d)]
    lib.fc_batch_info.argtypes = [vp, P(i), P(ll), P(ll), P(i)]
    lib.fc_batch_profile_enable.argtypes = [vp, i]
    lib.fc_batch_profile_read.argtypes = [vp, i, P(ll), P(d), P(d)]
    lib.fc_batch_sync.argtypes = [vp]
    lib.fc_batch_last_error.restype = C.c_char_p
    lib.fc_batch_last_error.argtypes = [vp]
    lib.fc_batch_destroy.argtypes = [vp]
    for name in EXPORTS:
        if name not in ("fc_last_error", "fc_footprint_estimate", "fc_batch_last_error"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _grid(prob) -> FcGrid:
    g = FcGrid()
    g.dim = prob.dim
    for k in range(3):
        g.n[k] = int(prob.n[k]) if k < prob.dim else 1
        g.lo[k] = float(prob.lo[k]) if k < prob.dim else 0.0
        g.hi[k] = float(prob.hi[k]) if k < prob.dim else 1.0
    return g


TC = {"none": 0, "tf32": 1, "tf32x3": 2, "bf16": 3}


ELEMENT = {"q1": 0, "q2": 1}


def _options(prob, cache: str, prec: str, nu=None, dedup: int = 1, tc: str = "none",
             badcut_frac: float | None = None, element: str = "q1", galerkin: bool = False) -> FcOptions:
    o = FcOptions()
    load().fc_options_default(C.byref(o))
    o.eta, o.nitsche_beta, o.omega = prob.eta, prob.beta, prob.omega
    o.nu_pre, o.nu_post = (prob.nu_pre, prob.nu_post) if nu is None else nu
    o.quad_depth = prob.qdepth
    o.cache, o.prec = CACHE[cache], PREC[prec]
    o.fgmres_restart = prob.restart
    o.bc_preset, o.ubar = prob.preset, prob.ubar
    o.force_kind = prob.force_kind
    for k in range(3):
        o.force[k] = float(prob.force[k])
    o.dedup = int(dedup)
    o.tc = TC[tc]
    o.element = ELEMENT[element]
    o.galerkin = 1 if galerkin else 0
    o.amr_uniform = int(getattr(prob, "amr_uniform", -1))
    if badcut_frac is not None:
        o.badcut_frac = float(badcut_frac)
    return o


def launch_count() -> int:
    n = C.c_longlong()
    load().fc_launch_count(C.byref(n))
    return n.value


def probe_fma_rate(precision: str = "fp64"):
    """(FLOP/s, launch ms) of independent FMA chains on every SM of the
    current GPU (fc_probe_fma_rate)."""
    f, ms = C.c_double(), C.c_double()
    st = load().fc_probe_fma_rate({"fp64": 0, "fp32": 1}[precision], C.byref(f), C.byref(ms))
    if st != FC_OK:
        raise FcError(st, "fc_probe_fma_rate failed")
    return f.value, ms.value


def footprint_estimate(prob, cache="inverse", prec="fp64") -> int:
    return int(load().fc_footprint_estimate(C.byref(_grid(prob)), prob.nlevels,
                                            C.byref(_options(prob, cache, prec))))


class Solver:
    """A finite cell Stokes problem set up on the GPU (one fc_handle)."""

    def __init__(self, prob, cache: str = "inverse", prec: str = "fp64", stream=None, nu=None,
                 dedup: int = 1, tc: str = "none", badcut_frac: float | None = None, element: str = "q1",
                 galerkin: bool = False):
        import torch
        if not torch.cuda.is_available():
            raise FcError(-1, "libfc needs a CUDA GPU")
        self.torch = torch
        self.lib = load()
        self.prob = prob
        self.dim = prob.dim
        self.nd = prob.dim + 1
        self.nlevels = prob.nlevels
        self.cache, self.prec, self.element = cache, prec, element
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = torch.cuda.current_device()
        self._sizes = {}
        shapes = np.asarray(prob.shapes, dtype=np.float64).reshape(-1, 9)
        arr = (FcShape * max(1, len(shapes)))()
        for s, row in enumerate(shapes):
            arr[s].type = int(row[0])
            for k in range(3):
                arr[s].c[k] = row[1 + k]
                arr[s].r[k] = row[4 + k]
            arr[s].rot[0], arr[s].rot[1] = row[7], row[8]
        self._shapes = arr
        ls = FcLevelset(len(shapes), C.cast(arr, C.POINTER(FcShape)))
        self.h = C.c_void_p()
        st = self.lib.fc_setup(C.byref(self.h), C.byref(_grid(prob)), C.byref(ls), float(prob.alpha),
                               int(prob.nlevels),
                               C.byref(_options(prob, cache, prec, nu, dedup, tc, badcut_frac, element, galerkin)),
                               C.c_void_p(self.stream.cuda_stream))
        self._check(st)

    # ---------------------------------------------------------------- util
    def _check(self, st):
        if st != FC_OK:
            msg = self.lib.fc_last_error(self.h).decode() if self.h else ""
            raise FcError(st, msg)

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.lib.fc_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def ndof(self, level=None) -> int:
        lv = self.nlevels if level is None else int(level)
        if lv not in self._sizes:
            n = C.c_longlong()
            self._check(self.lib.fc_info(self.h, lv, C.byref(n), None, None))
            self._sizes[lv] = n.value
        return self._sizes[lv]

    def info(self, level=None):
        n, p = C.c_longlong(), C.c_longlong()
        parts = (C.c_size_t * 8)()
        self._check(self.lib.fc_info(self.h, self.nlevels if level is None else level,
                                     C.byref(n), C.byref(p), parts))
        return {"ndof": n.value, "npatch": p.value, "bytes": list(parts)}

    def zeros(self, level=None):
        return self.torch.zeros(self.ndof(level), dtype=self.torch.float64, device=f"cuda:{self.device}")

    def _dev(self, v, level, name):
        """A contiguous float64 copy (or view) of v on this solver's GPU,
        checked to hold the level's DoF count."""
        t = v if self.torch.is_tensor(v) else self.torch.as_tensor(np.asarray(v, dtype=np.float64))
        t = t.to(device=f"cuda:{self.device}", dtype=self.torch.float64).contiguous()
        return self._need(t, level, name)

    def _need(self, t, level, name):
        return check_device_vector(self.torch, t, self.ndof(level), self.device, name)

    @staticmethod
    def _ptr(t):
        return C.c_void_p(t.data_ptr())

    # ---------------------------------------------------------------- ABI calls
    def rhs(self):
        b = self.zeros()
        self._check(self.lib.fc_rhs(self.h, self._ptr(b)))
        return b

    def residual(self, x, b, level=None):
        lv = self.nlevels if level is None else level
        x, b = self._dev(x, lv, "x"), self._dev(b, lv, "b")
        r = self.zeros(lv)
        self._check(self.lib.fc_residual(self.h, lv, self._ptr(x), self._ptr(b), self._ptr(r)))
        return r

    def apply(self, x, level=None):
        lv = self.nlevels if level is None else level
        x = self._dev(x, lv, "x")
        y = self.zeros(lv)
        self._check(self.lib.fc_apply(self.h, lv, self._ptr(x), self._ptr(y)))
        return y

    def smooth(self, x, b, level=None, nsweeps=1):
        """Returns a new vector: x after ``nsweeps`` RA sweeps."""
        lv = self.nlevels if level is None else level
        xx = self._dev(x, lv, "x").clone()
        b = self._dev(b, lv, "b")
        self._check(self.lib.fc_smooth(self.h, lv, self._ptr(xx), self._ptr(b), int(nsweeps)))
        return xx

    def smooth_(self, x, b, level=None, nsweeps=1):
        """In-place smoother on device tensors (no copies)."""
        lv = self.nlevels if level is None else level
        self._need(x, lv, "x")
        self._need(b, lv, "b")
        self._check(self.lib.fc_smooth(self.h, lv, self._ptr(x), self._ptr(b), int(nsweeps)))
        return x

    def smooth_noalloc_(self, x, b, level=None, nsweeps=1):
        """In-place smoother that allocates nothing (static device scratch);
        returns the status code so callers can inspect rejections."""
        lv = self.nlevels if level is None else level
        self._need(x, lv, "x")
        self._need(b, lv, "b")
        return self.lib.fc_smooth_noalloc(self.h, lv, self._ptr(x), self._ptr(b), int(nsweeps))

    def restrict(self, r, level=None):
        lv = self.nlevels if level is None else level
        r = self._dev(r, lv, "r")
        bc = self.zeros(lv - 1)
        self._check(self.lib.fc_restrict(self.h, lv, self._ptr(r), self._ptr(bc)))
        return bc

    def prolong_add(self, e, x, level=None):
        lv = self.nlevels if level is None else level
        e = self._dev(e, lv - 1, "e")
        xx = self._dev(x, lv, "x").clone()
        self._check(self.lib.fc_prolong_add(self.h, lv, self._ptr(e), self._ptr(xx)))
        return xx

    def coarse_solve(self, b):
        b = self._dev(b, 1, "b")
        x = self.zeros(1)
        self._check(self.lib.fc_coarse_solve(self.h, self._ptr(b), self._ptr(x)))
        return x

    def vcycle(self, x, b):
        xx = self._dev(x, None, "x").clone()
        b = self._dev(b, None, "b")
        self._check(self.lib.fc_vcycle(self.h, self._ptr(xx), self._ptr(b)))
        return xx

    def solve(self, b, x0=None, rtol=None, maxit=200):
        """FGMRES + GMG; returns (x, iterations, true relative residual)."""
        b = self._dev(b, None, "b")
        x = self.zeros() if x0 is None else self._dev(x0, None, "x0").clone()
        its, rel = C.c_int(), C.c_double()
        st = self.lib.fc_solve(self.h, self._ptr(b), self._ptr(x),
                               float(self.prob.rtol if rtol is None else rtol), int(maxit),
                               C.byref(its), C.byref(rel))
        if st not in (FC_OK, FC_ERR_NOT_CONVERGED):
            self._check(st)
        return x, its.value, rel.value

    def gmg_solve(self, b, x0=None, reduction=1e-9, maxit=100):
        """Standalone V-cycles until the residual falls by ``reduction``;
        returns (x, cycles, achieved reduction)."""
        b = self._dev(b, None, "b")
        x = self.zeros() if x0 is None else self._dev(x0, None, "x0").clone()
        its, red = C.c_int(), C.c_double()
        st = self.lib.fc_gmg_solve(self.h, self._ptr(b), self._ptr(x), float(reduction), int(maxit),
                                   C.byref(its), C.byref(red))
        if st not in (FC_OK, FC_ERR_NOT_CONVERGED):
            self._check(st)
        return x, its.value, red.value

    def solve_host(self, b_host, x_host, rtol=None, maxit=200):
        """FGMRES + GMG from host buffers (numpy or pinned torch CPU tensors)."""
        def ptr(a, name, writable):
            check_host_vector(self.torch, a, self.ndof(), name, writable)
            if self.torch.is_tensor(a):
                return C.c_void_p(a.data_ptr())
            return a.ctypes.data_as(C.c_void_p)
        its, rel = C.c_int(), C.c_double()
        st = self.lib.fc_solve_host(self.h, ptr(b_host, "b_host", False), ptr(x_host, "x_host", True),
                                    float(self.prob.rtol if rtol is None else rtol), int(maxit),
                                    C.byref(its), C.byref(rel))
        if st not in (FC_OK, FC_ERR_NOT_CONVERGED):
            self._check(st)
        return its.value, rel.value

    def patch_rows(self, node: int, level=None):
        lv = self.nlevels if level is None else level
        if getattr(self.prob, "amr_uniform", -1) >= 0:   # adaptive: d + 1 owned rows x patch DoFs
            out = np.zeros((self.nd, len(self.patch_dofs(node, level))))
        elif self.element == "q2":          # Q2-Q1: owned rows x slots
            out = np.zeros((25, 2214)) if self.dim == 3 else np.zeros((9, 171))
        else:
            ns = 402 if self.dim == 3 else 59
            out = np.zeros((self.nd, ns))
        self._check(self.lib.fc_patch_rows(self.h, lv, int(node),
                                           out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def patch_dofs(self, node: int, level=None):
        """Adaptive grids: the DoFs of the patch of free node `node`."""
        lv = self.nlevels if level is None else level
        buf = np.zeros(2048, dtype=np.int64)
        n = C.c_int()
        self._check(self.lib.fc_patch_dofs(self.h, lv, int(node), buf.ctypes.data_as(C.POINTER(C.c_longlong)),
                                           len(buf), C.byref(n)))
        return buf[:n.value].copy()

    def profile(self, on: bool = True):
        self._check(self.lib.fc_profile_enable(self.h, 1 if on else 0))

    def profile_read(self, kind: int):
        n, ms, by = C.c_longlong(), C.c_double(), C.c_double()
        self._check(self.lib.fc_profile_read(self.h, int(kind), C.byref(n), C.byref(ms), C.byref(by)))
        return n.value, ms.value, by.value

    def sync(self):
        self._check(self.lib.fc_sync(self.h))


class Batch:
    """Many Solver problems smoothed, cycled and solved together
    (fc_batch_*).  Vectors are packed: every problem's finest-level vector
    back to back, problem p at ``offsets[p]:offsets[p+1]``."""

    def __init__(self, solvers, stream=None, tile=None):
        """tile = (lanes per patch, threads, CTAs per SM) builds the batch with
        that patch-apply tile (fc_batch_create_tiled) instead of timing the
        candidates (fc_batch_create)."""
        import torch
        self.torch = torch
        self.lib = load()
        self.solvers = list(solvers)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = torch.cuda.current_device()
        hs = (C.c_void_p * len(self.solvers))(*[s.h.value for s in self.solvers])
        self.b = C.c_void_p()
        if tile is None:
            st = self.lib.fc_batch_create(C.byref(self.b), hs, len(self.solvers), C.c_void_p(self.stream.cuda_stream))
        else:
            st = self.lib.fc_batch_create_tiled(C.byref(self.b), hs, len(self.solvers),
                                                C.c_void_p(self.stream.cuda_stream), *[int(v) for v in tile])
        self._check(st)
        off = (C.c_longlong * (len(self.solvers) + 1))()
        self._check(self.lib.fc_batch_offsets(self.b, off))
        self.offsets = [int(v) for v in off]

    def _check(self, st):
        if st != FC_OK:
            msg = self.lib.fc_batch_last_error(self.b).decode() if self.b else ""
            raise FcError(st, msg)

    def close(self):
        if getattr(self, "b", None) and self.b.value:
            self.lib.fc_batch_destroy(self.b)
            self.b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def ndof(self) -> int:
        return self.offsets[-1]

    def _need(self, t, name):
        return check_device_vector(self.torch, t, self.ndof, self.device, name)

    def _open(self):
        """The batch works on its solvers' device data: refuse to run once
        the batch or any of its solvers was closed."""
        if not (getattr(self, "b", None) and self.b.value):
            raise FcError(FC_ERR_INVALID, "the batch was closed")
        if not all(getattr(s, "h", None) and s.h.value for s in self.solvers):
            raise FcError(FC_ERR_INVALID, "a solver of this batch was closed")

    def pack(self, vectors):
        vectors = list(vectors)
        if len(vectors) != len(self.solvers):
            raise FcError(FC_ERR_INVALID, f"pack: {len(vectors)} vectors for {len(self.solvers)} problems")
        out = self.torch.empty(self.ndof, dtype=self.torch.float64, device=f"cuda:{self.device}")
        for p, v in enumerate(vectors):
            t = v if self.torch.is_tensor(v) else self.torch.as_tensor(np.asarray(v, dtype=np.float64))
            n = self.offsets[p + 1] - self.offsets[p]
            if t.numel() != n:
                raise FcError(FC_ERR_INVALID, f"pack: problem {p} needs {n} values, got {t.numel()}")
            out[self.offsets[p]:self.offsets[p + 1]] = t.reshape(-1).to(device=out.device, dtype=self.torch.float64)
        return out

    def unpack(self, packed):
        return [packed[self.offsets[p]:self.offsets[p + 1]] for p in range(len(self.solvers))]

    def rhs(self):
        return self.pack([s.rhs() for s in self.solvers])

    def tile(self):
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        self._check(self.lib.fc_batch_tile(self.b, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def set_tile(self, lanes_per_patch, threads, ctas_per_sm):
        self._check(self.lib.fc_batch_set_tile(self.b, int(lanes_per_patch), int(threads), int(ctas_per_sm)))

    def info(self):
        n, nd, npch, lv = C.c_int(), C.c_longlong(), C.c_longlong(), C.c_int()
        self._check(self.lib.fc_batch_info(self.b, C.byref(n), C.byref(nd), C.byref(npch), C.byref(lv)))
        return {"nprob": n.value, "ndof": nd.value, "npatch_finest": npch.value, "levels_max": lv.value}

    def smooth_(self, x, b, nsweeps=1):
        self._open()
        self._need(x, "x")
        self._need(b, "b")
        self._check(self.lib.fc_batch_smooth(self.b, C.c_void_p(x.data_ptr()), C.c_void_p(b.data_ptr()),
                                             int(nsweeps)))
        return x

    def vcycle_(self, x, b):
        self._open()
        self._need(x, "x")
        self._need(b, "b")
        self._check(self.lib.fc_batch_vcycle(self.b, C.c_void_p(x.data_ptr()), C.c_void_p(b.data_ptr())))
        return x

    def solve(self, b, x0=None, rtol=1e-8, maxit=200):
        """Per-problem FGMRES + GMG; returns (packed x, iterations, relres)."""
        self._open()
        self._need(b, "b")
        x = (self.torch.zeros(self.ndof, dtype=self.torch.float64, device=f"cuda:{self.device}") if x0 is None
             else self._need(x0, "x0").clone())
        n = len(self.solvers)
        its = (C.c_int * n)()
        rel = (C.c_double * n)()
        st = self.lib.fc_batch_solve(self.b, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), float(rtol),
                                     int(maxit), its, rel)
        if st not in (FC_OK, FC_ERR_NOT_CONVERGED):
            self._check(st)
        return x, list(its), list(rel)

    def solve_host(self, b_host, x_host, rtol=1e-8, maxit=200):
        """Per-problem solves from packed pinned host tensors; x_host holds x0
        and receives x.  Returns (iterations, relres)."""
        self._open()
        check_host_vector(self.torch, b_host, self.ndof, "b_host")
        check_host_vector(self.torch, x_host, self.ndof, "x_host", writable=True)
        n = len(self.solvers)
        its = (C.c_int * n)()
        rel = (C.c_double * n)()
        st = self.lib.fc_batch_solve_host(self.b, C.c_void_p(b_host.data_ptr()), C.c_void_p(x_host.data_ptr()),
                                          float(rtol), int(maxit), its, rel)
        if st not in (FC_OK, FC_ERR_NOT_CONVERGED):
            self._check(st)
        return list(its), list(rel)

    def profile(self, on: bool = True):
        self._check(self.lib.fc_batch_profile_enable(self.b, 1 if on else 0))

    def profile_read(self, kind: int):
        n, ms, by = C.c_longlong(), C.c_double(), C.c_double()
        self._check(self.lib.fc_batch_profile_read(self.b, int(kind), C.byref(n), C.byref(ms), C.byref(by)))
        return n.value, ms.value, by.value

    def sync(self):
        self._check(self.lib.fc_batch_sync(self.b))
