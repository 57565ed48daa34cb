"""ctypes wrapper of the plain FP64 CPU oracle (oracle/amg_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference arm. The CUDA product path never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "amg_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liboracle.so")
# A prebuilt oracle library to load instead (the mutation test points this at builds of the
# oracle with one planted mistake each, to show that the pins catch it); unset in normal use.
LIB_OVERRIDE_ENV = "AMG_ORACLE_LIB"

OK, ERR_INVALID_ARG, ERR_BAD_MATRIX, ERR_OOM, ERR_NOT_CONVERGED, ERR_BREAKDOWN = 0, 1, 2, 3, 5, 6

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc: -O2, no FMA contraction, IEEE division."""
    if os.environ.get(LIB_OVERRIDE_ENV):
        return os.environ[LIB_OVERRIDE_ENV]
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        compile_oracle(SRC, tmp)
        os.replace(tmp, LIB)
    return LIB


def compile_oracle(src: str, out: str):
    """gcc -O2, no FMA contraction, IEEE division: the flags every build of the oracle uses."""
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                           "-shared", "-std=c99", "-o", out, src, "-lm"])


class Opts(C.Structure):
    _fields_ = [("aux_level", C.c_int), ("coarsest_max", C.c_int), ("kcycle_n", C.c_int),
                ("max_iters", C.c_int), ("has_bbox", C.c_int), ("bbox", C.c_double * 4),
                ("no_factor", C.c_int), ("dim", C.c_int), ("zbox", C.c_double * 2),
                ("nu_pre", C.c_int), ("nu_post", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            ip = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
            L.oamg_setup.argtypes = [C.c_int, ip, ip, dp, dp, dp, C.POINTER(Opts), C.POINTER(P)]
            L.oamg_setup.restype = C.c_int
            L.oamg_setup3.argtypes = [C.c_int, ip, ip, dp, dp, dp, dp, C.POINTER(Opts),
                                      C.POINTER(P)]
            L.oamg_setup3.restype = C.c_int
            L.oamg_get_zbox.argtypes = [P, dp]
            L.oamg_get_zbox.restype = None
            L.oamg_dim.argtypes = [P]
            L.oamg_dim.restype = C.c_int
            L.oamg_level_t3.argtypes = [P, C.c_int, ip]
            L.oamg_level_t3.restype = C.c_int
            L.oamg_bin3.argtypes = [C.c_int, dp, dp, dp, dp, C.c_int, ip]
            L.oamg_bin3.restype = None
            L.oamg_auto_level3.argtypes = [C.c_longlong]
            L.oamg_auto_level3.restype = C.c_int
            L.oamg_solve.argtypes = [P, dp, C.c_double, dp, C.POINTER(C.c_int),
                                     C.POINTER(C.c_double)]
            L.oamg_solve.restype = C.c_int
            L.oamg_free.argtypes = [P]
            L.oamg_free.restype = None
            L.oamg_num_levels.argtypes = [P]
            L.oamg_num_levels.restype = C.c_int
            L.oamg_aux_level.argtypes = [P]
            L.oamg_aux_level.restype = C.c_int
            L.oamg_get_bbox.argtypes = [P, dp]
            L.oamg_get_bbox.restype = None
            L.oamg_level_info.argtypes = [P, C.c_int, ip]
            L.oamg_level_info.restype = C.c_int
            L.oamg_level_get.argtypes = [P, C.c_int] + [P] * 8
            L.oamg_level_get.restype = C.c_int
            for name in ("oamg_bhat", "oamg_btilde"):
                getattr(L, name).argtypes = [P, C.c_int, dp, dp]
                getattr(L, name).restype = C.c_int
            L.oamg_smooth.argtypes = [P, C.c_int, C.c_int, dp, dp]
            L.oamg_smooth.restype = C.c_int
            L.oamg_bin.argtypes = [C.c_int, dp, dp, dp, C.c_int, ip]
            L.oamg_bin.restype = None
            L.oamg_auto_level.argtypes = [C.c_longlong]
            L.oamg_auto_level.restype = C.c_int
            _lib = L
    return _lib


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"{what} failed with status {status}")
        self.status = status


def auto_level(N: int, dim: int = 2) -> int:
    return lib().oamg_auto_level3(N) if dim == 3 else lib().oamg_auto_level(N)


def bin_points3(x, y, z, bbox6, L) -> np.ndarray:
    x, y, z = _f64(x), _f64(y), _f64(z)
    cell = np.empty(len(x), np.int32)
    lib().oamg_bin3(len(x), x, y, z, _f64(bbox6), L, cell)
    return cell


def bin_points(x, y, bbox, L) -> np.ndarray:
    x, y = _f64(x), _f64(y)
    cell = np.empty(len(x), np.int32)
    lib().oamg_bin(len(x), x, y, _f64(bbox), L, cell)
    return cell


class Level:
    """One level of the oracle hierarchy, copied out to numpy."""

    def __init__(self, n, rowptr, col, val, t1, t2, color, perm, agg, cellw, span, m, t3=None):
        self.n, self.rowptr, self.col, self.val = n, rowptr, col, val
        self.t1, self.t2, self.color, self.perm, self.agg = t1, t2, color, perm, agg
        self.cellw, self.span, self.m, self.t3 = cellw, span, m, t3

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))


class Hierarchy:
    """Oracle setup (Sec. 3-4 of the paper) for one matrix + node coordinates."""

    def __init__(self, rowptr, col, val, x, y, aux_level=0, coarsest_max=64, kcycle_n=2,
                 max_iters=200, bbox=None, no_factor=False, z=None, nu_pre=1, nu_post=1):
        """z given: the octree (3D) variant; bbox then has 6 entries a1,b1,a2,b2,a3,b3.
        nu_pre / nu_post: Gauss-Seidel sweeps of the pre- / post-smoothing (reading R10)."""
        L = lib()
        self._keep = (_i32(rowptr), _i32(col), _f64(val), _f64(x), _f64(y))
        bb = tuple(bbox) if bbox is not None else (0.0,) * 6
        o = Opts(aux_level, coarsest_max, kcycle_n, max_iters, 0 if bbox is None else 1,
                 (C.c_double * 4)(*bb[:4]), int(no_factor), 3 if z is not None else 2,
                 (C.c_double * 2)(*(bb[4:6] if len(bb) >= 6 else (0.0, 0.0))), int(nu_pre),
                 int(nu_post))
        h = C.c_void_p()
        n = len(self._keep[0]) - 1
        if z is not None:
            self._keep = self._keep + (_f64(z),)
            st = L.oamg_setup3(n, *self._keep, C.byref(o), C.byref(h))
        else:
            st = L.oamg_setup(n, *self._keep, C.byref(o), C.byref(h))
        if st != OK:
            raise OracleError(st, "oamg_setup")
        self.h = h
        self.n = n

    @classmethod
    def from_problem(cls, prob, **kw):
        z = getattr(prob, "z", None)
        if z is not None:
            kw.setdefault("z", z)
        return cls(prob.rowptr, prob.col, prob.val, prob.x, prob.y, **kw)

    @property
    def dim(self) -> int:
        return lib().oamg_dim(self.h)

    @property
    def zbox(self) -> np.ndarray:
        b = np.empty(2)
        lib().oamg_get_zbox(self.h, b)
        return b

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().oamg_free(h)
            self.h = None

    @property
    def nlev(self) -> int:
        return lib().oamg_num_levels(self.h)

    @property
    def L(self) -> int:
        return lib().oamg_aux_level(self.h)

    @property
    def bbox(self) -> np.ndarray:
        b = np.empty(4)
        lib().oamg_get_bbox(self.h, b)
        return b

    def level(self, l: int) -> Level:
        info = np.empty(5, np.int32)
        st = lib().oamg_level_info(self.h, l, info)
        if st != OK:
            raise OracleError(st, "oamg_level_info")
        n, nnz, cellw, span, m = (int(v) for v in info)
        rowptr = np.empty(n + 1, np.int32)
        col = np.empty(nnz, np.int32)
        val = np.empty(nnz)
        t1 = np.empty(n, np.int32)
        t2 = np.empty(n, np.int32)
        color = np.empty(n, np.int32)
        perm = np.empty(n, np.int32)
        has_agg = l < self.nlev - 1
        agg = np.empty(n, np.int32) if has_agg else None
        ptr = lambda a: a.ctypes.data if a is not None else None  # noqa: E731
        lib().oamg_level_get(self.h, l, ptr(rowptr), ptr(col), ptr(val), ptr(t1), ptr(t2),
                             ptr(color), ptr(perm), ptr(agg))
        t3 = None
        if self.dim == 3:
            t3 = np.empty(n, np.int32)
            lib().oamg_level_t3(self.h, l, t3)
        return Level(n, rowptr, col, val, t1, t2, color, perm, agg, cellw, span, m, t3)

    def levels(self):
        return [self.level(l) for l in range(self.nlev)]

    def smooth(self, l, f, u, backward=False):
        u = _f64(u).copy()
        lib().oamg_smooth(self.h, l, int(backward), _f64(f), u)
        return u

    def bhat(self, l, f):
        z = np.empty(len(f))
        lib().oamg_bhat(self.h, l, _f64(f), z)
        return z

    def btilde(self, l, f):
        u = np.empty(len(f))
        lib().oamg_btilde(self.h, l, _f64(f), u)
        return u

    def solve(self, b, tol=1e-8):
        """Returns (x, iters, relres, status)."""
        x = np.empty(self.n)
        it = C.c_int()
        rr = C.c_double()
        st = lib().oamg_solve(self.h, _f64(b), tol, x, C.byref(it), C.byref(rr))
        return x, it.value, rr.value, st
