"""The C-ABI library builds for sm_103a and exports every function include/amg.h declares.

Runs without a GPU: loading the library and resolving symbols makes no CUDA call.
"""
import ctypes

import pytest

from paper_1209_5421_gb300 import amg, build


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_header_declares_the_boundary():
    names = amg.declared_functions()
    for required in ("amg_setup", "amg_solve", "amg_free", "amg_hierarchy_bytes",
                     "amg_status_string", "amg_options_default", "amg_apply_cycle",
                     "amg_smooth", "amg_level_export", "amg_csr_to_ell"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [f for f in amg.declared_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_status_strings_without_gpu(libpath):
    lib = amg.lib()
    for s in range(9):
        assert amg.status_string(s)
    assert amg.status_string(0) == "ok"
    assert "unknown" in amg.status_string(99)


def test_options_defaults(libpath):
    o = amg.Options()
    amg.lib().amg_options_default(ctypes.byref(o))
    assert (o.aux_level, o.coarsest_max, o.kcycle_n, o.max_iters, o.outer, o.cycle_prec) == \
        (0, 64, 2, 200, amg.OUTER_FCG, amg.FP64)


def test_setup_rejects_bad_arguments_before_touching_the_gpu(libpath):
    L = amg.lib()
    h = ctypes.c_void_p()
    A = amg.Csr(0, 0, None, None, None)
    assert L.amg_setup(ctypes.byref(A), None, None, None, None, ctypes.byref(h)) == amg.ERR_INVALID_ARG
    assert h.value is None
    assert L.amg_setup(None, None, None, None, None, None) == amg.ERR_INVALID_ARG


def test_batch_setup_rejects_bad_arguments_before_touching_the_gpu(libpath):
    L = amg.lib()
    b = ctypes.c_void_p()
    rp = (ctypes.c_int32 * 3)(0, 1, 2)
    cl = (ctypes.c_int32 * 2)(0, 1)
    vl = (ctypes.c_double * 2)(1.0, 1.0)
    xy = (ctypes.c_double * 2)(0.0, 1.0)
    A = amg.Csr(2, 2, ctypes.cast(rp, ctypes.c_void_p), ctypes.cast(cl, ctypes.c_void_p),
                ctypes.cast(vl, ctypes.c_void_p))
    xp = ctypes.cast(xy, ctypes.c_void_p)
    bad_offsets = [(0, 2, 2), (0, 1, 3), (1, 1, 2), (0, 2, 1)]  # empty, past n, not from 0, ...
    for offs in bad_offsets:
        ro = (ctypes.c_int64 * 3)(*offs)
        st = L.amg_batch_setup(2, ctypes.cast(ro, ctypes.c_void_p), ctypes.byref(A), xp, xp, None,
                               None, ctypes.byref(b))
        assert st == amg.ERR_INVALID_ARG, offs
        assert b.value is None
    ro = (ctypes.c_int64 * 3)(0, 1, 2)
    assert L.amg_batch_setup(0, ctypes.cast(ro, ctypes.c_void_p), ctypes.byref(A), xp, xp, None,
                             None, ctypes.byref(b)) == amg.ERR_INVALID_ARG
    o = amg.Options()
    L.amg_options_default(ctypes.byref(o))
    o.outer = amg.OUTER_FGMRES
    assert L.amg_batch_setup(2, ctypes.cast(ro, ctypes.c_void_p), ctypes.byref(A), xp, xp,
                             ctypes.byref(o), None, ctypes.byref(b)) == amg.ERR_UNSUPPORTED
    assert L.amg_batch_solve(None, None, 1e-8, None, None, None, None, None) == amg.ERR_INVALID_ARG
    assert L.amg_batch_set_teams(None, 0) == amg.ERR_INVALID_ARG
    assert L.amg_batch_teams(None, None) == amg.ERR_INVALID_ARG
    L.amg_batch_free(None)
