"""ctypes binding of the FP64 CPU oracle (fc_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline leg of bench.py.  The product library never imports it, and it
never imports the product library.

A ``Level`` is one uniform background grid of the multigrid hierarchy
(Sec. 3: levels l = 1..L, L finest).  ``MG`` couples levels for the V-cycle
and FGMRES.  Problems are passed in duck-typed (any object with the fields
dim, n, lo, hi, shapes, alpha, qdepth, nlevels, eta, beta, omega, nu_pre,
nu_post, preset, force_kind, force, ubar).

The environment variables FC_ORACLE_LIB and FC_ORACLE_Q2_LIB, when set,
name other builds of fc_oracle.c / fc_oracle_q2.c to load instead of the ones
built here; the planted-mistake tests use them to run the pins against
altered copies of the oracle.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fc_oracle.c")
_LIB = os.path.join(_HERE, "libfc_oracle.so")
_lock = threading.Lock()
_lib = None

PMAX = 402
OMAX = 4


def compile_source(src: str, out: str) -> None:
    """gcc of one oracle source into a shared library (plain C, OpenMP, no FP
    contraction)."""
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-o", out, src, "-lm"]
    subprocess.check_call(cmd)


def build(force: bool = False) -> str:
    """Compile fc_oracle.c next to this file (when it changed)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            compile_source(_SRC, tmp)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    alt = os.environ.get("FC_ORACLE_LIB")
    if alt:
        lib = C.CDLL(alt)
    else:
        build()
        lib = C.CDLL(_LIB)
    _lib = _declare(lib)
    return _lib


def _declare(lib):
    """ctypes signatures of the fc_oracle.c entry points (also in the
    libraries of the variants that include it)."""
    vp, d, i, l = C.c_void_p, C.c_double, C.c_int, C.c_long
    P = C.POINTER
    lib.or_level_new.restype = vp
    lib.or_level_new.argtypes = [i, P(C.c_int), P(d), P(d), i, P(d), d, i, d, d, d, i, i, P(d), d]
    lib.or_level_free.argtypes = [vp]
    for fn in ("or_ndof", "or_nnodes", "or_ncell", "or_nbpoints", "or_nnz"):
        getattr(lib, fn).restype = l
        getattr(lib, fn).argtypes = [vp]
    lib.or_phi.restype = d
    lib.or_phi.argtypes = [vp, P(d)]
    lib.or_cell_element.restype = i
    lib.or_cell_element.argtypes = [vp, l, P(d), P(d), P(d), P(d), P(d)]
    lib.or_precompute_cells.argtypes = [vp]
    lib.or_dof_rows.argtypes = [vp, l, P(C.c_long), P(d), P(d)]
    lib.or_assemble.argtypes = [vp]
    lib.or_csr_copy.argtypes = [vp, P(C.c_long), P(C.c_long), P(d), P(d), P(C.c_ubyte)]
    lib.or_residual.argtypes = [vp, P(d), P(d), P(d)]
    lib.or_apply.argtypes = [vp, P(d), P(d)]
    lib.or_patch_dofs.restype = i
    lib.or_patch_dofs.argtypes = [vp, l, P(C.c_long), P(C.c_int)]
    lib.or_patch_matrix.restype = i
    lib.or_patch_matrix.argtypes = [vp, l, P(d), P(C.c_long), P(C.c_int)]
    lib.or_patch_inverse_rows.restype = i
    lib.or_patch_inverse_rows.argtypes = [vp, l, P(C.c_long), P(C.c_int), P(d)]
    lib.or_dense_solve.restype = i
    lib.or_dense_solve.argtypes = [i, P(d), P(d)]
    lib.or_dense_solve_eq.restype = i
    lib.or_dense_solve_eq.argtypes = [i, P(d), P(d)]
    lib.or_build_inverse.restype = i
    lib.or_build_inverse.argtypes = [vp]
    lib.or_sweep.restype = i
    lib.or_sweep.argtypes = [vp, P(d), P(d), i, P(C.c_long)]
    lib.or_apply_patches.argtypes = [vp, P(d), P(d), l, P(C.c_long)]
    lib.or_owner_count.argtypes = [vp, P(C.c_int)]
    lib.or_prolong_add.argtypes = [vp, vp, P(d), P(d)]
    lib.or_restrict.argtypes = [vp, vp, P(d), P(d)]
    lib.or_galerkin.argtypes = [vp, vp]
    lib.or_mg_new.restype = vp
    lib.or_mg_new.argtypes = [i, P(vp), i, i, i]
    lib.or_mg_free.argtypes = [vp]
    lib.or_vcycle.argtypes = [vp, P(d), P(d)]
    lib.or_fgmres.restype = i
    lib.or_fgmres.argtypes = [vp, P(d), P(d), d, i, i, P(d), P(d)]
    lib.or_gmg_solve.restype = i
    lib.or_gmg_solve.argtypes = [vp, P(d), P(d), d, i, P(d)]
    lib.or_num_threads.restype = i
    lib.or_set_threads.argtypes = [i]
    lib.or_bpoints_copy.argtypes = [vp, P(d), P(d), P(d), P(C.c_long)]
    return lib


def _p(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t))


def num_threads() -> int:
    return _load().or_num_threads()


def set_threads(n: int) -> None:
    _load().or_set_threads(int(n))


def dense_solve(A: np.ndarray, b: np.ndarray, equilibrate: bool = True) -> np.ndarray:
    """The oracle's own LU with partial pivoting on a dense matrix (by default
    of the symmetrically equilibrated matrix, as in the local solves)."""
    lib = _load()
    a = np.ascontiguousarray(A, dtype=np.float64).copy()
    x = np.ascontiguousarray(b, dtype=np.float64).copy()
    fn = lib.or_dense_solve_eq if equilibrate else lib.or_dense_solve
    if fn(a.shape[0], _p(a), _p(x)) != 0:
        raise np.linalg.LinAlgError("singular")
    return x


class Level:
    """One grid level with its finite cell discretisation."""

    def __init__(self, dim, n, lo, hi, shapes, alpha, qdepth, eta=1e-3, beta=100.0,
                 omega=0.8, preset=0, force_kind=0, force=(0.0, 0.0, 0.0), ubar=0.3, lib=None):
        lib = _load() if lib is None else lib
        self.dim = int(dim)
        self.n = tuple(int(k) for k in n)
        nn = (C.c_int * 3)(*(list(self.n) + [1] * (3 - self.dim)))
        lo_ = (C.c_double * 3)(*(list(lo) + [0.0] * (3 - self.dim)))
        hi_ = (C.c_double * 3)(*(list(hi) + [1.0] * (3 - self.dim)))
        sh = np.ascontiguousarray(np.asarray(shapes, dtype=np.float64).reshape(-1, 9))
        self._shapes = sh
        fo = (C.c_double * 3)(*list(force))
        self.h = lib.or_level_new(self.dim, nn, lo_, hi_, sh.shape[0], _p(sh), float(alpha),
                                  int(qdepth), float(eta), float(beta), float(omega), int(preset),
                                  int(force_kind), fo, float(ubar))
        self.lib = lib
        self.ndof = lib.or_ndof(self.h)
        self.nnodes = lib.or_nnodes(self.h)
        self.ncell = lib.or_ncell(self.h)
        self.ndpn = self.dim + 1
        self._assembled = False

    @classmethod
    def from_problem(cls, prob, level=None):
        lvl = prob.nlevels if level is None else level
        return cls(prob.dim, prob.level_n(lvl), prob.lo, prob.hi, prob.shapes, prob.alpha,
                   prob.qdepth, prob.eta, prob.beta, prob.omega, prob.preset, prob.force_kind,
                   prob.force, prob.ubar)

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.lib.or_level_free(self.h)
                self.h = None
        except Exception:
            pass

    # geometry / elements -------------------------------------------------
    def phi(self, x):
        xx = (C.c_double * 3)(*(list(x) + [0.0] * (3 - len(x))))
        return self.lib.or_phi(self.h, xx)

    def cell_element(self, cell: int):
        nl = 1 << self.dim
        A = np.zeros((nl, nl)); B = np.zeros((self.dim, nl, nl)); Cm = np.zeros((nl, nl))
        f = np.zeros((self.dim, nl)); st = np.zeros(4)
        if self.lib.or_cell_element(self.h, int(cell), _p(A), _p(B), _p(Cm), _p(f), _p(st)) != 0:
            raise IndexError(f"cell {cell} out of range")
        return {"A": A, "B": B, "C": Cm, "f": f, "fluid_volume": st[0],
                "boundary_measure": st[1], "nvol": int(st[2]), "nbnd": int(st[3])}

    def bpoints(self):
        n = self.lib.or_nbpoints(self.h)
        x = np.zeros((n, 3)); nr = np.zeros((n, 3)); w = np.zeros(n); c = np.zeros(n, dtype=np.int64)
        if n:
            self.lib.or_bpoints_copy(self.h, _p(x), _p(nr), _p(w), _p(c, C.c_long))
        return x, nr, w, c

    def precompute_cells(self):
        self.lib.or_precompute_cells(self.h)

    # operator --------------------------------------------------------------
    def assemble(self):
        if not self._assembled:
            self.lib.or_assemble(self.h)
            self._assembled = True

    def csr(self):
        import scipy.sparse as sp
        self.assemble()
        nnz = self.lib.or_nnz(self.h)
        rp = np.zeros(self.ndof + 1, dtype=np.int64); col = np.zeros(nnz, dtype=np.int64)
        val = np.zeros(nnz); rhs = np.zeros(self.ndof); fixed = np.zeros(self.ndof, dtype=np.uint8)
        self.lib.or_csr_copy(self.h, _p(rp, C.c_long), _p(col, C.c_long), _p(val), _p(rhs),
                             _p(fixed, C.c_ubyte))
        return sp.csr_matrix((val, col, rp), shape=(self.ndof, self.ndof)), rhs, fixed.astype(bool)

    def dof_rows(self, dofs):
        """Rows of the eliminated operator for the given DoFs: array
        [len(dofs), 3^d, d+1] over the neighbour nodes, and their b values."""
        d = np.ascontiguousarray(dofs, dtype=np.int64)
        nnb = 27 if self.dim == 3 else 9
        rows = np.zeros((len(d), nnb, self.ndpn)); rhs = np.zeros(len(d))
        self.lib.or_dof_rows(self.h, len(d), _p(d, C.c_long), _p(rows), _p(rhs))
        return rows, rhs

    def residual(self, b, x):
        self.assemble()
        r = np.zeros(self.ndof)
        b = np.ascontiguousarray(b, dtype=np.float64); x = np.ascontiguousarray(x, dtype=np.float64)
        self.lib.or_residual(self.h, _p(b), _p(x), _p(r))
        return r

    def apply(self, x):
        self.assemble()
        y = np.zeros(self.ndof)
        x = np.ascontiguousarray(x, dtype=np.float64)
        self.lib.or_apply(self.h, _p(x), _p(y))
        return y

    # patches and the smoother ---------------------------------------------
    def patch_dofs(self, node: int):
        d = np.zeros(PMAX, dtype=np.int64); own = np.zeros(OMAX, dtype=np.int32)
        n = self.lib.or_patch_dofs(self.h, int(node), _p(d, C.c_long), _p(own, C.c_int))
        return d[:n].copy(), own.copy()

    def patch_matrix(self, node: int):
        d = np.zeros(PMAX, dtype=np.int64); own = np.zeros(OMAX, dtype=np.int32)
        Li = np.zeros(PMAX * PMAX)
        n = self.lib.or_patch_matrix(self.h, int(node), _p(Li), _p(d, C.c_long), _p(own, C.c_int))
        return Li[: n * n].reshape(n, n).copy(), d[:n].copy(), own.copy()

    def patch_inverse_rows(self, node: int):
        d = np.zeros(PMAX, dtype=np.int64); own = np.zeros(OMAX, dtype=np.int32)
        rows = np.zeros((OMAX, PMAX))
        n = self.lib.or_patch_inverse_rows(self.h, int(node), _p(d, C.c_long), _p(own, C.c_int),
                                           _p(rows))
        if n < 0:
            raise np.linalg.LinAlgError("singular patch")
        return rows[:, :n].copy(), d[:n].copy(), own.copy()

    def build_inverse(self):
        self.assemble()
        return self.lib.or_build_inverse(self.h)

    def sweep(self, b, x, mode: int = 0, order=None):
        """One RA smoother sweep; returns the new x (input not modified)."""
        self.assemble()
        xx = np.ascontiguousarray(x, dtype=np.float64).copy()
        b = np.ascontiguousarray(b, dtype=np.float64)
        o = None
        if order is not None:
            order = np.ascontiguousarray(order, dtype=np.int64)
            o = _p(order, C.c_long)
        bad = self.lib.or_sweep(self.h, _p(b), _p(xx), int(mode), o)
        if bad:
            raise np.linalg.LinAlgError(f"{bad} singular patches")
        return xx

    def apply_patches(self, r, x, patches):
        self.assemble()
        xx = np.ascontiguousarray(x, dtype=np.float64).copy()
        r = np.ascontiguousarray(r, dtype=np.float64)
        pl = np.ascontiguousarray(patches, dtype=np.int64)
        self.lib.or_apply_patches(self.h, _p(r), _p(xx), len(pl), _p(pl, C.c_long))
        return xx

    def owner_count(self):
        cnt = np.zeros(self.ndof, dtype=np.int32)
        self.lib.or_owner_count(self.h, _p(cnt, C.c_int))
        return cnt


def prolong_add(fine: Level, coarse: Level, ec, xf):
    fine.assemble(); coarse.assemble()
    out = np.ascontiguousarray(xf, dtype=np.float64).copy()
    ec = np.ascontiguousarray(ec, dtype=np.float64)
    fine.lib.or_prolong_add(fine.h, coarse.h, _p(ec), _p(out))
    return out


def restrict(fine: Level, coarse: Level, rf):
    fine.assemble(); coarse.assemble()
    bc = np.zeros(coarse.ndof)
    rf = np.ascontiguousarray(rf, dtype=np.float64)
    fine.lib.or_restrict(fine.h, coarse.h, _p(rf), _p(bc))
    return bc


class MG:
    """Multigrid hierarchy of a problem: levels[0] coarsest .. levels[-1] finest."""

    def __init__(self, prob=None, levels=None, nu_pre=None, nu_post=None, mode: int = 0,
                 galerkin: bool = False):
        if levels is None:
            levels = [Level.from_problem(prob, l) for l in range(1, prob.nlevels + 1)]
        self.levels = levels
        if galerkin:
            # coarse operators R L_f P from the finest level down (or_galerkin)
            for lv in levels:
                lv.assemble()
            for l in range(len(levels) - 2, -1, -1):
                levels[l].lib.or_galerkin(levels[l].h, levels[l + 1].h)
        self.nu_pre = prob.nu_pre if nu_pre is None and prob is not None else (nu_pre or 0)
        self.nu_post = prob.nu_post if nu_post is None and prob is not None else (nu_post or 0)
        arr = (C.c_void_p * len(levels))(*[lv.h for lv in levels])
        for lv in levels:
            lv._assembled = True
        self.lib = levels[0].lib
        self.h = self.lib.or_mg_new(len(levels), arr, int(self.nu_pre), int(self.nu_post), int(mode))
        self.fine = levels[-1]

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.lib.or_mg_free(self.h)
                self.h = None
        except Exception:
            pass

    def rhs(self):
        _, b, _ = self.fine.csr()
        return b

    def vcycle(self, x, b):
        xx = np.ascontiguousarray(x, dtype=np.float64).copy()
        b = np.ascontiguousarray(b, dtype=np.float64)
        self.lib.or_vcycle(self.h, _p(xx), _p(b))
        return xx

    def fgmres(self, b, x0=None, rtol=1e-8, maxit=200, restart=30):
        n = self.fine.ndof
        x = np.zeros(n) if x0 is None else np.ascontiguousarray(x0, dtype=np.float64).copy()
        b = np.ascontiguousarray(b, dtype=np.float64)
        rel = np.zeros(1); hist = np.zeros(maxit + 1)
        its = self.lib.or_fgmres(self.h, _p(b), _p(x), float(rtol), int(maxit), int(restart),
                                 _p(rel), _p(hist))
        return x, its, float(rel[0]), hist[:its].copy()

    def gmg_solve(self, b, x0=None, reduction=1e-9, maxit=100):
        n = self.fine.ndof
        x = np.zeros(n) if x0 is None else np.ascontiguousarray(x0, dtype=np.float64).copy()
        b = np.ascontiguousarray(b, dtype=np.float64)
        rel = np.zeros(1)
        its = self.lib.or_gmg_solve(self.h, _p(b), _p(x), float(reduction), int(maxit), _p(rel))
        return x, its, float(rel[0])


# ---------------------------------------------------------------------------
# Q2-Q1 (Taylor-Hood) variant with the lower-corner ownership rule
# (fc_oracle_q2.c, which includes fc_oracle.c)
_SRC_Q2 = os.path.join(_HERE, "fc_oracle_q2.c")
_LIB_Q2 = os.path.join(_HERE, "libfc_oracle_q2.so")
_lib_q2 = None
Q2PMAX = 2214
Q2OMAX = 25


def build_q2(force: bool = False) -> str:
    """Compile fc_oracle_q2.c next to this file (when it or fc_oracle.c changed)."""
    with _lock:
        stale = (not os.path.exists(_LIB_Q2) or os.path.getmtime(_LIB_Q2) < os.path.getmtime(_SRC_Q2)
                 or os.path.getmtime(_LIB_Q2) < os.path.getmtime(_SRC))
        if force or stale:
            tmp = _LIB_Q2 + f".tmp{os.getpid()}"
            compile_source(_SRC_Q2, tmp)
            os.replace(tmp, _LIB_Q2)
    return _LIB_Q2


def _load_q2():
    global _lib_q2
    if _lib_q2 is not None:
        return _lib_q2
    alt = os.environ.get("FC_ORACLE_Q2_LIB")
    if alt:
        lib = C.CDLL(alt)
    else:
        build_q2()
        lib = C.CDLL(_LIB_Q2)
    vp, d, i, l = C.c_void_p, C.c_double, C.c_int, C.c_long
    P = C.POINTER
    lib.q2_level_new.restype = vp
    lib.q2_level_new.argtypes = [i, P(C.c_int), P(d), P(d), i, P(d), d, i, d, d, d, i, i, P(d), d]
    lib.q2_level_free.argtypes = [vp]
    for fn in ("q2_ndof", "q2_nv", "q2_np", "q2_nnz"):
        getattr(lib, fn).restype = l
        getattr(lib, fn).argtypes = [vp]
    lib.q2_cell_element.restype = i
    lib.q2_cell_element.argtypes = [vp, l, P(d), P(d), P(d), P(d)]
    lib.q2_assemble.argtypes = [vp]
    lib.q2_csr_copy.argtypes = [vp, P(C.c_long), P(C.c_long), P(d), P(d), P(C.c_ubyte)]
    lib.q2_apply.argtypes = [vp, P(d), P(d)]
    lib.q2_residual.argtypes = [vp, P(d), P(d), P(d)]
    lib.q2_patch_dofs.restype = i
    lib.q2_patch_dofs.argtypes = [vp, l, P(C.c_long), P(C.c_int)]
    lib.q2_patch_matrix.restype = i
    lib.q2_patch_matrix.argtypes = [vp, l, P(d), P(C.c_long), P(C.c_int)]
    lib.q2_patch_inverse_rows.restype = i
    lib.q2_patch_inverse_rows.argtypes = [vp, l, P(C.c_long), P(C.c_int), P(d)]
    lib.q2_build_inverse.restype = i
    lib.q2_build_inverse.argtypes = [vp]
    lib.q2_sweep.restype = i
    lib.q2_sweep.argtypes = [vp, P(d), P(d), P(C.c_long)]
    lib.q2_owner_count.argtypes = [vp, P(C.c_int)]
    lib.q2_prolong_add.argtypes = [vp, vp, P(d), P(d)]
    lib.q2_restrict.argtypes = [vp, vp, P(d), P(d)]
    lib.q2_mg_new.restype = vp
    lib.q2_mg_new.argtypes = [i, P(vp), i, i]
    lib.q2_mg_free.argtypes = [vp]
    lib.q2_vcycle.argtypes = [vp, P(d), P(d)]
    lib.q2_fgmres.restype = i
    lib.q2_fgmres.argtypes = [vp, P(d), P(d), d, i, i, P(d)]
    lib.q2_gmg_solve.restype = i
    lib.q2_gmg_solve.argtypes = [vp, P(d), P(d), d, i, P(d)]
    _lib_q2 = lib
    return lib


class Q2Level:
    """One grid level with the Q2-Q1 discretisation.  DoFs: velocity at the
    Q2 nodes ((2 n_k + 1) per direction, x fastest, d components inner), then
    the pressure at the vertices."""

    def __init__(self, dim, n, lo, hi, shapes, alpha, qdepth, eta=1e-3, beta=100.0, omega=0.8, preset=0,
                 force_kind=0, force=(0.0, 0.0, 0.0), ubar=0.3):
        lib = _load_q2()
        self.lib = lib
        self.dim = int(dim)
        self.n = tuple(int(k) for k in n)
        nn = (C.c_int * 3)(*(list(self.n) + [1] * (3 - self.dim)))
        lo_ = (C.c_double * 3)(*(list(lo) + [0.0] * (3 - self.dim)))
        hi_ = (C.c_double * 3)(*(list(hi) + [1.0] * (3 - self.dim)))
        sh = np.ascontiguousarray(np.asarray(shapes, dtype=np.float64).reshape(-1, 9))
        self._shapes = sh
        fo = (C.c_double * 3)(*list(force))
        self.h = lib.q2_level_new(self.dim, nn, lo_, hi_, sh.shape[0], _p(sh), float(alpha), int(qdepth),
                                  float(eta), float(beta), float(omega), int(preset), int(force_kind), fo,
                                  float(ubar))
        self.ndof = lib.q2_ndof(self.h)
        self.nv = lib.q2_nv(self.h)
        self.np = lib.q2_np(self.h)
        self.ncell = int(np.prod(self.n))
        self._assembled = False

    @classmethod
    def from_problem(cls, prob, level=None):
        lvl = prob.nlevels if level is None else level
        return cls(prob.dim, prob.level_n(lvl), prob.lo, prob.hi, prob.shapes, prob.alpha, prob.qdepth,
                   prob.eta, prob.beta, prob.omega, prob.preset, prob.force_kind, prob.force, prob.ubar)

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.lib.q2_level_free(self.h)
                self.h = None
        except Exception:
            pass

    def cell_element(self, cell: int):
        na = 27 if self.dim == 3 else 9
        nb = 1 << self.dim
        A = np.zeros((na, na)); B = np.zeros((self.dim, na, nb)); f = np.zeros((self.dim, na)); st = np.zeros(4)
        if self.lib.q2_cell_element(self.h, int(cell), _p(A), _p(B), _p(f), _p(st)) != 0:
            raise IndexError(f"cell {cell} out of range")
        return {"A": A, "B": B, "f": f, "fluid_volume": st[0], "boundary_measure": st[1],
                "nvol": int(st[2]), "nbnd": int(st[3])}

    def assemble(self):
        if not self._assembled:
            self.lib.q2_assemble(self.h)
            self._assembled = True

    def csr(self):
        import scipy.sparse as sp
        self.assemble()
        nnz = self.lib.q2_nnz(self.h)
        rp = np.zeros(self.ndof + 1, dtype=np.int64); col = np.zeros(nnz, dtype=np.int64)
        val = np.zeros(nnz); rhs = np.zeros(self.ndof); fixed = np.zeros(self.ndof, dtype=np.uint8)
        self.lib.q2_csr_copy(self.h, _p(rp, C.c_long), _p(col, C.c_long), _p(val), _p(rhs), _p(fixed, C.c_ubyte))
        return sp.csr_matrix((val, col, rp), shape=(self.ndof, self.ndof)), rhs, fixed.astype(bool)

    def residual(self, b, x):
        self.assemble()
        r = np.zeros(self.ndof)
        self.lib.q2_residual(self.h, _p(np.ascontiguousarray(b, dtype=np.float64)),
                             _p(np.ascontiguousarray(x, dtype=np.float64)), _p(r))
        return r

    def apply(self, x):
        self.assemble()
        y = np.zeros(self.ndof)
        self.lib.q2_apply(self.h, _p(np.ascontiguousarray(x, dtype=np.float64)), _p(y))
        return y

    def patch_dofs(self, vert: int):
        self.assemble()
        d = np.zeros(Q2PMAX, dtype=np.int64); own = np.zeros(Q2OMAX, dtype=np.int32)
        n = self.lib.q2_patch_dofs(self.h, int(vert), _p(d, C.c_long), _p(own, C.c_int))
        return d[:n].copy(), own.copy()

    def patch_matrix(self, vert: int):
        self.assemble()
        d = np.zeros(Q2PMAX, dtype=np.int64); own = np.zeros(Q2OMAX, dtype=np.int32)
        Li = np.zeros(Q2PMAX * Q2PMAX)
        n = self.lib.q2_patch_matrix(self.h, int(vert), _p(Li), _p(d, C.c_long), _p(own, C.c_int))
        return Li[: n * n].reshape(n, n).copy(), d[:n].copy(), own.copy()

    def patch_inverse_rows(self, vert: int):
        self.assemble()
        d = np.zeros(Q2PMAX, dtype=np.int64); own = np.zeros(Q2OMAX, dtype=np.int32)
        rows = np.zeros((Q2OMAX, Q2PMAX))
        n = self.lib.q2_patch_inverse_rows(self.h, int(vert), _p(d, C.c_long), _p(own, C.c_int), _p(rows))
        if n < 0:
            raise np.linalg.LinAlgError("singular patch")
        return rows[:, :n].copy(), d[:n].copy(), own.copy()

    def sweep(self, b, x, order=None):
        self.assemble()
        xx = np.ascontiguousarray(x, dtype=np.float64).copy()
        o = None
        if order is not None:
            order = np.ascontiguousarray(order, dtype=np.int64)
            o = _p(order, C.c_long)
        self.lib.q2_sweep(self.h, _p(np.ascontiguousarray(b, dtype=np.float64)), _p(xx), o)
        return xx

    def owner_count(self):
        self.assemble()
        cnt = np.zeros(self.ndof, dtype=np.int32)
        self.lib.q2_owner_count(self.h, _p(cnt, C.c_int))
        return cnt


def q2_prolong_add(fine: Q2Level, coarse: Q2Level, ec, xf):
    fine.assemble(); coarse.assemble()
    out = np.ascontiguousarray(xf, dtype=np.float64).copy()
    fine.lib.q2_prolong_add(fine.h, coarse.h, _p(np.ascontiguousarray(ec, dtype=np.float64)), _p(out))
    return out


def q2_restrict(fine: Q2Level, coarse: Q2Level, rf):
    fine.assemble(); coarse.assemble()
    bc = np.zeros(coarse.ndof)
    fine.lib.q2_restrict(fine.h, coarse.h, _p(np.ascontiguousarray(rf, dtype=np.float64)), _p(bc))
    return bc


class Q2MG:
    """Q2-Q1 multigrid hierarchy: levels[0] coarsest .. levels[-1] finest."""

    def __init__(self, prob=None, levels=None, nu_pre=None, nu_post=None):
        if levels is None:
            levels = [Q2Level.from_problem(prob, l) for l in range(1, prob.nlevels + 1)]
        self.levels = levels
        self.nu_pre = prob.nu_pre if nu_pre is None else nu_pre
        self.nu_post = prob.nu_post if nu_post is None else nu_post
        for lv in levels:
            lv._assembled = True
        self.lib = levels[0].lib
        arr = (C.c_void_p * len(levels))(*[lv.h for lv in levels])
        self.h = self.lib.q2_mg_new(len(levels), arr, int(self.nu_pre), int(self.nu_post))
        self.fine = levels[-1]

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.lib.q2_mg_free(self.h)
                self.h = None
        except Exception:
            pass

    def rhs(self):
        _, b, _ = self.fine.csr()
        return b

    def vcycle(self, x, b):
        xx = np.ascontiguousarray(x, dtype=np.float64).copy()
        self.lib.q2_vcycle(self.h, _p(xx), _p(np.ascontiguousarray(b, dtype=np.float64)))
        return xx

    def fgmres(self, b, x0=None, rtol=1e-8, maxit=200, restart=30):
        n = self.fine.ndof
        x = np.zeros(n) if x0 is None else np.ascontiguousarray(x0, dtype=np.float64).copy()
        rel = np.zeros(1)
        its = self.lib.q2_fgmres(self.h, _p(np.ascontiguousarray(b, dtype=np.float64)), _p(x), float(rtol),
                                 int(maxit), int(restart), _p(rel))
        return x, its, float(rel[0])

    def gmg_solve(self, b, x0=None, reduction=1e-9, maxit=100):
        n = self.fine.ndof
        x = np.zeros(n) if x0 is None else np.ascontiguousarray(x0, dtype=np.float64).copy()
        rel = np.zeros(1)
        its = self.lib.q2_gmg_solve(self.h, _p(np.ascontiguousarray(b, dtype=np.float64)), _p(x), float(reduction),
                                    int(maxit), _p(rel))
        return x, its, float(rel[0])


# ---------------------------------------------------------------------------
# Adaptive space-tree grids, quadtrees and octrees (fc_oracle_amr.c, which includes fc_oracle.c)
_SRC_AMR = os.path.join(_HERE, "fc_oracle_amr.c")
_LIB_AMR = os.path.join(_HERE, "libfc_oracle_amr.so")
_lib_amr = None


def build_amr(force: bool = False) -> str:
    """Compile fc_oracle_amr.c next to this file (when it or fc_oracle.c changed)."""
    with _lock:
        stale = (not os.path.exists(_LIB_AMR) or os.path.getmtime(_LIB_AMR) < os.path.getmtime(_SRC_AMR)
                 or os.path.getmtime(_LIB_AMR) < os.path.getmtime(_SRC))
        if force or stale:
            tmp = _LIB_AMR + f".tmp{os.getpid()}"
            compile_source(_SRC_AMR, tmp)
            os.replace(tmp, _LIB_AMR)
    return _LIB_AMR


def _load_amr():
    global _lib_amr
    if _lib_amr is not None:
        return _lib_amr
    alt = os.environ.get("FC_ORACLE_AMR_LIB")
    if alt:
        lib = C.CDLL(alt)
    else:
        build_amr()
        lib = C.CDLL(_LIB_AMR)
    _declare(lib)
    vp, i, l = C.c_void_p, C.c_int, C.c_long
    P = C.POINTER
    lib.amr_tree_fine.restype = vp
    lib.amr_tree_fine.argtypes = [vp, P(C.c_int), i, i]
    lib.amr_tree_coarsen.restype = vp
    lib.amr_tree_coarsen.argtypes = [vp]
    lib.amr_tree_free.argtypes = [vp]
    lib.amr_tree_level.restype = i
    lib.amr_tree_level.argtypes = [vp, i, i, i]
    lib.amr_level_new.restype = vp
    lib.amr_level_new.argtypes = [vp, P(vp), vp]
    lib.amr_free_nodes.restype = l
    lib.amr_free_nodes.argtypes = [vp, P(l)]
    lib.amr_hanging.restype = l
    lib.amr_hanging.argtypes = [vp, P(l), P(i), P(l)]
    lib.amr_patch_rows.restype = i
    lib.amr_patch_rows.argtypes = [vp, l, P(l), P(i), P(C.c_double), i]
    lib.amr_patch_stride.restype = i
    lib.amr_patch_stride.argtypes = [vp]
    lib.amr_prolongation.restype = l
    lib.amr_prolongation.argtypes = [vp, P(l), P(l), P(C.c_double)]
    _lib_amr = lib
    return lib


class AMRLevel(Level):
    """One level of an adaptive space-tree hierarchy (quadtree in 2D, octree
    in 3D): an or_level whose operator, patches and prolongation
    fc_oracle_amr.c built.  DoFs: the free nodes in lattice order (x fastest,
    then y, then z), the velocity components and then p per node."""

    def __init__(self, handle, tree, lib, lattice_n, dim=2):
        self.lib = lib
        self.h = handle
        self.tree = tree
        self.dim = dim
        self.n = tuple(lattice_n)
        self.ndof = lib.or_ndof(handle)
        self.nnodes = lib.or_nnodes(handle)
        self.ndpn = dim + 1
        self._assembled = True

    def patch_inverse_rows(self, vert: int):
        cap = self.lib.amr_patch_stride(self.h)
        d = np.zeros(cap, dtype=np.int64); own = np.zeros(OMAX, dtype=np.int32)
        rows = np.zeros((OMAX, cap))
        n = self.lib.amr_patch_rows(self.h, int(vert), _p(d, C.c_long), _p(own, C.c_int), _p(rows), cap)
        return rows[:, :n].copy(), d[:n].copy(), own.copy()

    def patch_dofs(self, vert: int):
        _, d, own = self.patch_inverse_rows(vert)
        return d, own

    def free_vertices(self):
        n = self.lib.amr_free_nodes(self.tree, None)
        v = np.zeros(n, dtype=np.int64)
        self.lib.amr_free_nodes(self.tree, _p(v, C.c_long))
        return v

    def hanging(self):
        """Hanging lattice vertices and their parents: (n, 2) in 2D (edge
        midpoints); in 3D (n, 4) with -1 after the two parents of an edge
        midpoint (face centres have four)."""
        n = self.lib.amr_hanging(self.tree, None, None, None)
        v = np.zeros(n, dtype=np.int64); npar = np.zeros(n, dtype=np.int32)
        par = np.zeros((n, 4), dtype=np.int64)
        self.lib.amr_hanging(self.tree, _p(v, C.c_long), _p(npar, C.c_int), _p(par, C.c_long))
        return v, (par[:, :2].copy() if self.dim == 2 else par)

    def leaf_levels(self):
        """Leaf level of every lattice cell: [y][x] in 2D, [z][y][x] in 3D."""
        if self.dim == 2:
            nx, ny = self.n
            return np.array([[self.lib.amr_tree_level(self.tree, x, y, 0) for x in range(nx)] for y in range(ny)])
        nx, ny, nz = self.n
        return np.array([[[self.lib.amr_tree_level(self.tree, x, y, z) for x in range(nx)] for y in range(ny)]
                         for z in range(nz)])

    def prolongation(self):
        import scipy.sparse as sp
        nnz = self.lib.amr_prolongation(self.h, None, None, None)
        if nnz < 0:
            return None
        rp = np.zeros(self.nnodes + 1, dtype=np.int64); col = np.zeros(nnz, dtype=np.int64)
        val = np.zeros(nnz)
        self.lib.amr_prolongation(self.h, _p(rp, C.c_long), _p(col, C.c_long), _p(val))
        return sp.csr_matrix((val, col, rp), shape=(self.nnodes, int(col.max()) + 1 if nnz else 0))

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.lib.or_level_free(self.h)
                self.h = None
            if getattr(self, "tree", None):
                self.lib.amr_tree_free(self.tree)
                self.tree = None
        except Exception:
            pass


def amr_levels(prob):
    """The adaptive hierarchy of a problem with prob.amr_uniform = U >= 0:
    lattice prob.n (the cells of the finest level), root grid
    prob.n / 2^(L-1), every cell refined uniformly to level U, cut cells to
    level L-1, 2:1 balanced; coarser levels by Algorithm 1.  Returns the
    AMRLevel objects, coarsest first."""
    assert prob.dim in (2, 3) and prob.amr_uniform >= 0
    lib = _load_amr()
    L = prob.nlevels
    R = L - 1
    root = [k >> R for k in prob.n]
    uni = [Level(prob.dim, tuple(k << r for k in root), prob.lo, prob.hi, prob.shapes, prob.alpha, prob.qdepth,
                 prob.eta, prob.beta, prob.omega, prob.preset, prob.force_kind, prob.force, prob.ubar, lib=lib)
           for r in range(R + 1)]
    uarr = (C.c_void_p * len(uni))(*[u.h for u in uni])
    nr = (C.c_int * 3)(*(list(root) + [1] * (3 - len(root))))
    trees = [lib.amr_tree_fine(uni[R].h, nr, int(prob.amr_uniform), R)]
    for _ in range(R):
        trees.append(lib.amr_tree_coarsen(trees[-1]))
    trees = trees[::-1]  # coarsest first
    levels = []
    for l in range(L):
        h = lib.amr_level_new(trees[l], uarr, trees[l - 1] if l > 0 else None)
        if not h:
            raise RuntimeError("adaptive level construction failed (patch or adjacency overflow)")
        levels.append(AMRLevel(h, trees[l], lib, prob.n, dim=prob.dim))
    for lv in levels:
        lv._uniform = uni  # keep the element data alive
    return levels


class AMRMG(MG):
    """Multigrid on the adaptive hierarchy: fc_oracle.c's V-cycle, FGMRES and
    standalone GMG with the adaptive levels."""

    def __init__(self, prob):
        super().__init__(prob, levels=amr_levels(prob))
