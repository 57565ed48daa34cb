"""Python binding of libamg_gb300.so (include/amg.h): argument marshalling only.

Every step of setup and solve runs in the library's CUDA kernels. Arrays may be numpy
arrays (host memory; the library stages them to the device) or torch tensors (device or
host memory). There is no CPU fallback: if the library is missing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# AMG_GB300_LIBRARY selects another build of the library (the bounds-checking variant
# libamg_gb300_bc.so in its tests)
LIB_PATH = os.environ.get("AMG_GB300_LIBRARY") or os.path.join(HERE, "libamg_gb300.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "amg.h")

OK = 0
ERR_INVALID_ARG, ERR_BAD_MATRIX, ERR_OOM, ERR_CUDA = 1, 2, 3, 4
ERR_NOT_CONVERGED, ERR_BREAKDOWN, ERR_TIMEOUT, ERR_UNSUPPORTED = 5, 6, 7, 8
OUTER_FCG, OUTER_FGMRES = 0, 1
FP64, FP32 = 0, 1


class AmgError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: status {status}")
        self.status = status


class Csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("aux_level", C.c_int), ("coarsest_max", C.c_int), ("kcycle_n", C.c_int),
                ("max_iters", C.c_int), ("outer", C.c_int), ("cycle_prec", C.c_int),
                ("fgmres_restart", C.c_int), ("has_bbox", C.c_int), ("bbox", C.c_double * 4),
                ("zbox", C.c_double * 2), ("nu_pre", C.c_int), ("nu_post", C.c_int)]


_lib = None


def declared_functions() -> list[str]:
    """Names of the functions include/amg.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(amg_[a-z0-9_]+)\s*\(", text)))


def lib():
    """Load libamg_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1209_5421_gb300.build`")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        L.amg_options_default.argtypes = [C.POINTER(Options)]
        L.amg_options_default.restype = None
        L.amg_setup.argtypes = [C.POINTER(Csr), P, P, C.POINTER(Options), P, C.POINTER(P)]
        L.amg_solve.argtypes = [P, P, C.c_double, P, C.POINTER(C.c_int), C.POINTER(C.c_double), P]
        L.amg_hierarchy_bytes.argtypes = [P, C.POINTER(C.c_size_t)]
        L.amg_free.argtypes = [P]
        L.amg_free.restype = None
        L.amg_status_string.argtypes = [C.c_int]
        L.amg_status_string.restype = C.c_char_p
        L.amg_last_error.argtypes = []
        L.amg_last_error.restype = C.c_char_p
        L.amg_num_levels.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.amg_get_bbox.argtypes = [P, P]
        L.amg_setup3.argtypes = [C.POINTER(Csr), P, P, P, C.POINTER(Options), P, C.POINTER(P)]
        L.amg_setup3.restype = C.c_int
        L.amg_get_box3.argtypes = [P, P, P]
        L.amg_get_box3.restype = C.c_int
        L.amg_level_t3.argtypes = [P, C.c_int, P]
        L.amg_level_t3.restype = C.c_int
        L.amg_level_info.argtypes = [P, C.c_int, P]
        L.amg_level_export.argtypes = [P, C.c_int] + [P] * 7
        L.amg_apply_cycle.argtypes = [P, C.c_int, P, P, P]
        L.amg_smooth.argtypes = [P, C.c_int, C.c_int, P, P, P]
        L.amg_csr_to_ell.argtypes = [C.c_int32, P, P, P, C.c_int32, C.c_int, P, P, P]
        L.amg_csr_to_ell_noalloc.argtypes = [C.c_int32, P, P, P, C.c_int32, C.c_int, P, P, P]
        L.amg_launch_counts.argtypes = [P, P, P]
        L.amg_profile_enable.argtypes = [P, C.c_int]
        L.amg_profile_read.argtypes = [P, C.c_int, P, P, P, P, P, C.POINTER(C.c_int)]
        L.amg_kernel_name.argtypes = [C.c_int]
        L.amg_kernel_name.restype = C.c_char_p
        L.amg_batch_setup.argtypes = [C.c_int32, P, C.POINTER(Csr), P, P, C.POINTER(Options), P,
                                      C.POINTER(P)]
        L.amg_batch_solve.argtypes = [P, P, C.c_double, P, P, P, P, P]
        L.amg_batch_create.argtypes = [C.c_int32, P, C.c_int32, P, C.POINTER(P)]
        L.amg_batch_create.restype = C.c_int
        L.amg_batch_info.argtypes = [P, P, P, P, P, P]
        L.amg_batch_timeline.argtypes = [P, P, P]
        L.amg_batch_timeline.restype = C.c_int
        L.amg_batch_set_teams.argtypes = [P, C.c_int32]
        L.amg_batch_set_teams.restype = C.c_int
        L.amg_batch_teams.argtypes = [P, P]
        L.amg_batch_teams.restype = C.c_int
        L.amg_batch_system.argtypes = [P, C.c_int32]
        L.amg_batch_system.restype = P
        L.amg_batch_moved_bytes.argtypes = [P, C.POINTER(C.c_double)]
        L.amg_setup_many.argtypes = [C.c_int32, P, C.POINTER(Csr), P, P, C.POINTER(Options), P, P]
        L.amg_batch_free.argtypes = [P]
        L.amg_batch_free.restype = None
        for f in ("amg_batch_setup", "amg_batch_solve", "amg_batch_info"):
            getattr(L, f).restype = C.c_int
        for f in ("amg_setup", "amg_solve", "amg_hierarchy_bytes", "amg_num_levels",
                  "amg_get_bbox", "amg_level_info", "amg_level_export", "amg_apply_cycle",
                  "amg_smooth", "amg_csr_to_ell", "amg_csr_to_ell_noalloc", "amg_launch_counts",
                  "amg_profile_enable",
                  "amg_profile_read"):
            getattr(L, f).restype = C.c_int
        L.amg_debug_barrier_fault.argtypes = [P, C.c_int64, C.c_int32]
        L.amg_debug_barrier_fault.restype = C.c_int
        L.amg_debug_batch_barrier_fault.argtypes = [P, C.c_int64, C.c_int32]
        L.amg_debug_batch_barrier_fault.restype = C.c_int
        L.amg_debug_fail_allocation.argtypes = [C.c_int64]
        L.amg_debug_fail_allocation.restype = C.c_int
        L.amg_debug_pool_bytes_in_use.argtypes = [C.c_int32, C.POINTER(C.c_int64)]
        L.amg_debug_pool_bytes_in_use.restype = C.c_int
        L.amg_debug_bounds_flags.argtypes = [C.POINTER(C.c_int32)]
        L.amg_debug_bounds_flags.restype = C.c_int
        _lib = L
    return _lib


def debug_fail_allocation(k: int):
    """Make the k-th device allocation of the library from now on fail (0: disarm)."""
    _check(lib().amg_debug_fail_allocation(int(k)), "amg_debug_fail_allocation")


def bounds_flags() -> int:
    """Index-check flags of the bounds-checking build since the last call (raises
    AmgError(ERR_UNSUPPORTED) in the normal build)."""
    v = C.c_int32()
    _check(lib().amg_debug_bounds_flags(C.byref(v)), "amg_debug_bounds_flags")
    return v.value


def pool_bytes_in_use(device: int = 0) -> int:
    """Bytes allocated from the device's default memory pool (the library's allocations)."""
    v = C.c_int64()
    _check(lib().amg_debug_pool_bytes_in_use(int(device), C.byref(v)),
           "amg_debug_pool_bytes_in_use")
    return v.value


def _ptr(a) -> int | None:
    """Raw address of a numpy array or torch tensor (must be contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(stream) -> int | None:
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _check(status: int, what: str):
    if status != OK:
        raise AmgError(status, f"{what}: {lib().amg_last_error().decode()}")


_TORCH_DTYPE = {np.dtype(np.int32): "torch.int32", np.dtype(np.float64): "torch.float64"}


def _is_tensor(a) -> bool:
    return hasattr(a, "data_ptr") and not isinstance(a, np.ndarray)


def _count(a) -> int:
    return int(a.numel()) if _is_tensor(a) else int(a.size)


def _as(a, dtype, n=None, what="array"):
    """An input array for a C call. numpy arrays (and other array-likes) become contiguous
    arrays of `dtype`; a torch tensor is passed as it is and must already have that dtype (the
    library reads its bytes as `dtype`). n: the number of entries the call reads. A raw
    pointer carries no length, so a shorter buffer would be read past its end: checked here."""
    if _is_tensor(a):
        if str(a.dtype) != _TORCH_DTYPE[np.dtype(dtype)]:
            raise TypeError(f"{what}: a tensor of {a.dtype}; the library reads "
                            f"{_TORCH_DTYPE[np.dtype(dtype)]}")
    else:
        a = np.ascontiguousarray(a, dtype=dtype)
    if n is not None and _count(a) != n:
        raise ValueError(f"{what}: {_count(a)} entries, expected {n}")
    return a


def _out(a, dtype, n, what):
    """A caller-provided output buffer (written in place, so never converted): `n` entries of
    `dtype`, contiguous."""
    if _is_tensor(a):
        if str(a.dtype) != _TORCH_DTYPE[np.dtype(dtype)]:
            raise TypeError(f"{what}: a tensor of {a.dtype}, expected "
                            f"{_TORCH_DTYPE[np.dtype(dtype)]}")
    elif not isinstance(a, np.ndarray) or a.dtype != np.dtype(dtype):
        raise TypeError(f"{what}: expected a numpy array or tensor of {np.dtype(dtype)}")
    if _count(a) != n:
        raise ValueError(f"{what}: {_count(a)} entries, expected {n}")
    return a


def status_string(s: int) -> str:
    return lib().amg_status_string(s).decode()


class Hierarchy:
    """amg_setup / amg_solve on one matrix with node coordinates (paper Sec. 3-4)."""

    def __init__(self, rowptr, col, val, x, y, aux_level=0, coarsest_max=64, kcycle_n=2,
                 max_iters=200, cycle_prec=FP64, outer=OUTER_FCG, fgmres_restart=30,
                 bbox=None, stream=None, z=None, nu_pre=1, nu_post=1):
        """z given: the octree (3D) variant (amg_setup3); bbox then has 6 entries.
        nu_pre / nu_post: Gauss-Seidel sweeps of the pre- / post-smoothing."""
        L = lib()
        rp = _as(rowptr, np.int32, what="rowptr")
        n = _count(rp) - 1
        if n < 0:
            raise ValueError("rowptr: no entries (a CSR matrix of n rows has n + 1)")
        cl = _as(col, np.int32, what="col")
        nnz = _count(cl)
        vl = _as(val, np.float64, nnz, "val")
        xx, yy = _as(x, np.float64, n, "x"), _as(y, np.float64, n, "y")
        zz = _as(z, np.float64, n, "z") if z is not None else None
        self._keep = (rp, cl, vl, xx, yy, zz)  # alive until the call returns
        A = Csr(n, nnz, _ptr(rp), _ptr(cl), _ptr(vl))
        o = Options()
        L.amg_options_default(C.byref(o))
        o.aux_level, o.coarsest_max, o.kcycle_n, o.max_iters = aux_level, coarsest_max, kcycle_n, max_iters
        o.cycle_prec, o.outer, o.fgmres_restart = cycle_prec, outer, fgmres_restart
        o.nu_pre, o.nu_post = nu_pre, nu_post
        if bbox is not None:
            o.has_bbox = 1
            for k in range(4):
                o.bbox[k] = bbox[k]
            if len(bbox) >= 6:
                o.zbox[0], o.zbox[1] = bbox[4], bbox[5]
        h = C.c_void_p()
        if zz is not None:
            st = L.amg_setup3(C.byref(A), _ptr(xx), _ptr(yy), _ptr(zz), C.byref(o),
                              _stream(stream), C.byref(h))
        else:
            st = L.amg_setup(C.byref(A), _ptr(xx), _ptr(yy), C.byref(o), _stream(stream),
                             C.byref(h))
        self._keep = None
        _check(st, "amg_setup")
        self.h = h
        self.n = n

    @classmethod
    def from_problem(cls, prob, **kw):
        if getattr(prob, "z", None) is not None:
            kw.setdefault("z", prob.z)
        return cls(prob.rowptr, prob.col, prob.val, prob.x, prob.y, **kw)

    def close(self):
        if getattr(self, "h", None):
            if not getattr(self, "_view", False):
                lib().amg_free(self.h)
            self.h = None

    @classmethod
    def view(cls, handle: int, n: int, owner):
        """A Hierarchy over a handle owned elsewhere (a batch's system): never freed here;
        `owner` is kept alive while the view is."""
        self = cls.__new__(cls)
        self.h = C.c_void_p(handle)
        self.n = n
        self._view = True
        self._owner = owner
        return self

    @property
    def dim(self) -> int:
        d = C.c_int()
        _check(lib().amg_get_box3(self.h, C.byref(d), None), "amg_get_box3")
        return d.value

    @property
    def box3(self) -> np.ndarray:
        b = np.empty(6)
        _check(lib().amg_get_box3(self.h, None, _ptr(b)), "amg_get_box3")
        return b

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, b, tol=1e-8, x=None, stream=None, check=False):
        """x = A^{-1} b. Returns (x, iters, relres, status). x: numpy if b is numpy."""
        b = _as(b, np.float64, self.n, "b")
        if x is None:
            x = np.empty(self.n) if isinstance(b, np.ndarray) else b.new_empty(self.n)
        else:
            _out(x, np.float64, self.n, "x")
        it = C.c_int()
        rr = C.c_double()
        st = lib().amg_solve(self.h, _ptr(b), tol, _ptr(x), C.byref(it), C.byref(rr),
                             _stream(stream))
        if check or st not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
            _check(st, "amg_solve")
        return x, it.value, rr.value, st

    @property
    def nbytes(self) -> int:
        v = C.c_size_t()
        _check(lib().amg_hierarchy_bytes(self.h, C.byref(v)), "amg_hierarchy_bytes")
        return v.value

    @property
    def nlev(self) -> int:
        n = C.c_int()
        a = C.c_int()
        _check(lib().amg_num_levels(self.h, C.byref(n), C.byref(a)), "amg_num_levels")
        return n.value

    @property
    def L(self) -> int:
        n = C.c_int()
        a = C.c_int()
        _check(lib().amg_num_levels(self.h, C.byref(n), C.byref(a)), "amg_num_levels")
        return a.value

    @property
    def bbox(self) -> np.ndarray:
        b = np.empty(4)
        _check(lib().amg_get_bbox(self.h, _ptr(b)), "amg_get_bbox")
        return b

    def level_info(self, l: int) -> dict:
        info = np.zeros(8, np.int64)
        _check(lib().amg_level_info(self.h, l, _ptr(info)), "amg_level_info")
        keys = ("n", "stored", "cellw", "span", "m", "padded", "coarsest", "nblocks")
        return dict(zip(keys, (int(v) for v in info)))

    def level(self, l: int) -> dict:
        """Natural-order host copies of level l: agg, color, t1, t2 and the CSR operator."""
        inf = self.level_info(l)
        n, nnz = inf["n"], inf["stored"]
        out = {k: np.empty(n, np.int32) for k in ("agg", "color", "t1", "t2")}
        out["rowptr"] = np.empty(n + 1, np.int32)
        out["col"] = np.empty(nnz, np.int32)
        out["val"] = np.empty(nnz)
        _check(lib().amg_level_export(self.h, l, _ptr(out["agg"]), _ptr(out["color"]),
                                      _ptr(out["t1"]), _ptr(out["t2"]), _ptr(out["rowptr"]),
                                      _ptr(out["col"]), _ptr(out["val"])), "amg_level_export")
        if self.dim == 3:
            out["t3"] = np.empty(n, np.int32)
            _check(lib().amg_level_t3(self.h, l, _ptr(out["t3"])), "amg_level_t3")
        out.update(inf)
        return out

    def launch_counts(self) -> tuple[int, int]:
        s = np.zeros(1, np.int64)
        v = np.zeros(1, np.int64)
        _check(lib().amg_launch_counts(self.h, _ptr(s), _ptr(v)), "amg_launch_counts")
        return int(s[0]), int(v[0])

    def debug_barrier_fault(self, limit_ns: int = 0, extra: int = 0):
        """Host-set barrier fault of the cycle kernel for the following solves (0, 0: off)."""
        _check(lib().amg_debug_barrier_fault(self.h, int(limit_ns), int(extra)),
               "amg_debug_barrier_fault")

    def profile(self, enable: bool | int = True):
        """0/False: off; 1/True: per-kernel and per-op timing, tail ops one by one; 2: the
        same with the shared-memory tail timed as a whole (no per-op work added to it)."""
        _check(lib().amg_profile_enable(self.h, int(enable)), "amg_profile_enable")

    def profile_read(self) -> list[dict]:
        cap = 256
        kind = np.zeros(cap, np.int32)
        level = np.zeros(cap, np.int32)
        launches = np.zeros(cap, np.int64)
        ms = np.zeros(cap)
        by = np.zeros(cap)
        cnt = C.c_int()
        _check(lib().amg_profile_read(self.h, cap, _ptr(kind), _ptr(level), _ptr(launches),
                                      _ptr(ms), _ptr(by), C.byref(cnt)), "amg_profile_read")
        out = []
        for k in range(min(cnt.value, cap)):
            nm = lib().amg_kernel_name(int(kind[k])).decode()
            out.append({"name": f"{nm}@L{int(level[k])}", "kind": nm, "level": int(level[k]),
                        "launches": int(launches[k]), "ms": float(ms[k]), "bytes": float(by[k])})
        return out

    def apply_cycle(self, level: int, f, stream=None):
        f = _as(f, np.float64, self.level_info(level)["n"], "f")
        z = np.empty(_count(f)) if isinstance(f, np.ndarray) else f.new_empty(_count(f))
        _check(lib().amg_apply_cycle(self.h, level, _ptr(f), _ptr(z), _stream(stream)),
               "amg_apply_cycle")
        return z

    def smooth(self, level: int, f, u, backward=False, stream=None):
        n = self.level_info(level)["n"]
        f = _as(f, np.float64, n, "f")
        u = _as(u, np.float64, n, "u").copy()
        _check(lib().amg_smooth(self.h, level, int(backward), _ptr(f), _ptr(u), _stream(stream)),
               "amg_smooth")
        return u


def csr_to_ell(rowptr, col, val, width, diag_first=True, stream=None):
    """The paper's ELL format (Sec. 4.1): column-major Aj (cols, -1 pad), Ax (vals, 0 pad)."""
    rowptr, col = _as(rowptr, np.int32, what="rowptr"), _as(col, np.int32, what="col")
    val = _as(val, np.float64, _count(col), "val")
    rows = _count(rowptr) - 1
    if isinstance(rowptr, np.ndarray) and rows >= 0:  # the packer trusts rowptr: check it
        if rowptr[0] != 0 or (np.diff(rowptr) < 0).any() or rowptr[-1] > _count(col):
            raise ValueError("rowptr must rise from 0 to at most len(col)")
    Aj = np.empty(rows * width, np.int32)
    Ax = np.empty(rows * width)
    _check(lib().amg_csr_to_ell(rows, _ptr(rowptr), _ptr(col), _ptr(val), width,
                                int(diag_first), _ptr(Aj), _ptr(Ax), _stream(stream)),
           "amg_csr_to_ell")
    return Aj, Ax


def concatenate(problems, device=None):
    """The block-diagonal CSR of many systems, the layout amg_batch_setup takes.

    problems: list of (rowptr, col, val, x, y) of each system (local indexing, host arrays).
    Returns (row_off, rowptr, col, val, x, y): row_off (host int64, one entry per system and
    the total) and the concatenated arrays, as torch tensors on `device` if one is given."""
    sizes = [len(p[0]) - 1 for p in problems]
    nnzs = [len(p[1]) for p in problems]
    for k, p in enumerate(problems):
        if sizes[k] < 0 or len(p[2]) != nnzs[k] or len(p[3]) != sizes[k] \
                or len(p[4]) != sizes[k]:
            raise ValueError(f"system {k}: rowptr needs n + 1 entries, val as many as col, "
                             "x and y n each")
    row_off = np.zeros(len(problems) + 1, np.int64)
    row_off[1:] = np.cumsum(sizes)
    nz_off = np.zeros(len(problems) + 1, np.int64)
    nz_off[1:] = np.cumsum(nnzs)
    if row_off[-1] >= 2**31 or nz_off[-1] >= 2**31:
        raise ValueError("the concatenation needs fewer than 2^31 rows and entries")
    rp = np.empty(row_off[-1] + 1, np.int32)
    cl = np.empty(nz_off[-1], np.int32)
    vl = np.empty(nz_off[-1], np.float64)
    xx = np.empty(row_off[-1], np.float64)
    yy = np.empty(row_off[-1], np.float64)
    for k, p in enumerate(problems):
        r0, r1, z0, z1 = row_off[k], row_off[k + 1], nz_off[k], nz_off[k + 1]
        np.add(np.asarray(p[0])[:-1], z0, out=rp[r0:r1], casting="unsafe")
        np.add(np.asarray(p[1]), r0, out=cl[z0:z1], casting="unsafe")
        vl[z0:z1] = p[2]
        xx[r0:r1] = p[3]
        yy[r0:r1] = p[4]
    rp[-1] = nz_off[-1]
    arrays = [rp, cl, vl, xx, yy]
    if device is not None:
        import torch

        arrays = [torch.as_tensor(a).to(device) for a in arrays]
    return (row_off, *arrays)


def setup_many(problems=None, concatenated=None, stream=None, device=None, **kw):
    """amg_setup_many: one Hierarchy per system, all set up together (problems or
    concatenated as for Batch; the options of Hierarchy). Each is freed on its own."""
    L = lib()
    if concatenated is None:
        concatenated = concatenate(problems, device)
    row_off, rp, cl, vl, xx, yy = concatenated
    row_off = np.asarray(row_off, np.int64)
    nprob = len(row_off) - 1
    A = Csr(int(row_off[-1]), len(cl), _ptr(rp), _ptr(cl), _ptr(vl))
    o = Options()
    L.amg_options_default(C.byref(o))
    for k, v in kw.items():
        if k == "bbox":
            o.has_bbox = 1
            for j in range(4):
                o.bbox[j] = v[j]
        elif k == "outer":
            o.outer = v
        elif k in ("aux_level", "coarsest_max", "kcycle_n", "max_iters", "cycle_prec",
                   "fgmres_restart", "nu_pre", "nu_post"):
            setattr(o, k, v)
        else:
            raise TypeError(f"unknown option {k!r}")
    out = (C.c_void_p * nprob)()
    _check(L.amg_setup_many(nprob, row_off.ctypes.data, C.byref(A), _ptr(xx), _ptr(yy),
                            C.byref(o), _stream(stream), C.cast(out, C.c_void_p)),
           "amg_setup_many")
    hs = []
    for p in range(nprob):
        h = Hierarchy.__new__(Hierarchy)
        h.h = C.c_void_p(out[p])
        h.n = int(row_off[p + 1] - row_off[p])
        h._keep = None
        hs.append(h)
    return hs


class Batch:
    """amg_batch_setup / amg_batch_solve: many independent systems, one persistent kernel.

    problems: list of (rowptr, col, val, x, y) of each system (local indexing, host arrays);
    they are concatenated into one block-diagonal CSR here (the layout the C ABI takes).
    concatenated: the output of `concatenate` instead of problems (the systems laid out
    already, on the host or the device).
    """

    def __init__(self, problems=None, aux_level=0, coarsest_max=64, kcycle_n=2, max_iters=200,
                 cycle_prec=FP64, stream=None, device=None, nu_pre=1, nu_post=1,
                 concatenated=None, bbox=None):
        L = lib()
        if concatenated is None:
            concatenated = concatenate(problems, device)
        row_off, rp, cl, vl, xx, yy = concatenated
        row_off = np.asarray(row_off, np.int64)
        self.row_off = row_off
        self.n = int(row_off[-1])
        self.nprob = len(row_off) - 1
        A = Csr(self.n, len(cl), _ptr(rp), _ptr(cl), _ptr(vl))
        o = Options()
        L.amg_options_default(C.byref(o))
        o.aux_level, o.coarsest_max, o.kcycle_n, o.max_iters = aux_level, coarsest_max, kcycle_n, max_iters
        o.cycle_prec, o.outer = cycle_prec, OUTER_FCG
        o.nu_pre, o.nu_post = nu_pre, nu_post
        if bbox is not None:  # one auxiliary box for every system
            o.has_bbox = 1
            for k in range(4):
                o.bbox[k] = bbox[k]
        b = C.c_void_p()
        st = L.amg_batch_setup(self.nprob, row_off.ctypes.data, C.byref(A), _ptr(xx), _ptr(yy),
                               C.byref(o), _stream(stream), C.byref(b))
        _check(st, "amg_batch_setup")
        self.b = b

    @classmethod
    def from_problems(cls, probs, **kw):
        return cls([(p.rowptr, p.col, p.val, p.x, p.y) for p in probs], **kw)

    @classmethod
    def over(cls, hierarchies, threads=0, stream=None):
        """A batch over existing Hierarchy objects (borrowed: keep them alive)."""
        self = cls.__new__(cls)
        hs = (C.c_void_p * len(hierarchies))(*[h.h for h in hierarchies])
        b = C.c_void_p()
        _check(lib().amg_batch_create(len(hierarchies), C.cast(hs, C.c_void_p), threads,
                                      _stream(stream), C.byref(b)), "amg_batch_create")
        self.b = b
        self.nprob = len(hierarchies)
        sizes = [h.n for h in hierarchies]
        self.row_off = np.zeros(self.nprob + 1, np.int64)
        self.row_off[1:] = np.cumsum(sizes)
        self.n = int(self.row_off[-1])
        self._borrowed = list(hierarchies)
        return self

    def set_teams(self, max_team: int):
        """amg_batch_set_teams: 0 = teams sized per system, 1 = one CTA per system, k = at
        most k CTAs per system."""
        _check(lib().amg_batch_set_teams(self.b, int(max_team)), "amg_batch_set_teams")

    def teams(self) -> np.ndarray:
        """amg_batch_teams: CTAs of each system's team in the launch shape in use."""
        t = np.zeros(self.nprob, np.int32)
        _check(lib().amg_batch_teams(self.b, t.ctypes.data), "amg_batch_teams")
        return t

    def close(self):
        if getattr(self, "b", None):
            lib().amg_batch_free(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, rhs, tol=1e-8, x=None, stream=None):
        """All systems: rhs concatenated (numpy or device tensor). Returns (x, iters, relres,
        status) with per-system numpy arrays; the call's own status is max-severity first."""
        rhs = _as(rhs, np.float64, self.n, "rhs")
        if x is None:
            x = np.empty(self.n) if isinstance(rhs, np.ndarray) else rhs.new_empty(self.n)
        else:
            _out(x, np.float64, self.n, "x")
        it = np.zeros(self.nprob, np.int32)
        rr = np.zeros(self.nprob, np.float64)
        st = np.zeros(self.nprob, np.int32)
        r = lib().amg_batch_solve(self.b, _ptr(rhs), tol, _ptr(x), it.ctypes.data,
                                  rr.ctypes.data, st.ctypes.data, _stream(stream))
        # per-system outcomes come back in `status`; other failures raise
        if r not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN, ERR_TIMEOUT):
            _check(r, "amg_batch_solve")
        return x, it, rr, st

    def system(self, p: int) -> "Hierarchy":
        """System p's hierarchy (owned by the batch) as a non-owning Hierarchy view."""
        h = lib().amg_batch_system(self.b, int(p))
        if not h:
            raise AmgError(ERR_INVALID_ARG, f"no system {p}")
        return Hierarchy.view(h, int(self.row_off[p + 1] - self.row_off[p]), self)

    def debug_barrier_fault(self, limit_ns: int = 0, extra: int = 0):
        """Host-set fault of the team barriers for the following solves (0, 0: off)."""
        _check(lib().amg_debug_batch_barrier_fault(self.b, int(limit_ns), int(extra)),
               "amg_debug_batch_barrier_fault")

    def info(self) -> dict:
        n = C.c_int32()
        t = C.c_int32()
        c = C.c_int32()
        ms = (C.c_double * 4)()
        nb = C.c_size_t()
        _check(lib().amg_batch_info(self.b, C.byref(n), C.byref(t), C.byref(c), ms, C.byref(nb)),
               "amg_batch_info")
        return {"nprob": n.value, "threads": t.value, "ctas": c.value,
                "tuned_ms": list(ms), "bytes": nb.value}

    def moved_bytes(self) -> float:
        """amg_batch_moved_bytes: algorithmic bytes the last solve moved (its roofline)."""
        v = C.c_double()
        _check(lib().amg_batch_moved_bytes(self.b, C.byref(v)), "amg_batch_moved_bytes")
        return v.value

    def timeline(self):
        """(start_ns, end_ns) of every system in the last solve, after the earliest start."""
        a = np.zeros(self.nprob, np.int64)
        e = np.zeros(self.nprob, np.int64)
        _check(lib().amg_batch_timeline(self.b, a.ctypes.data, e.ctypes.data), "amg_batch_timeline")
        return a, e
