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
