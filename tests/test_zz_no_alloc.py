"""amg_csr_to_ell_noalloc: the allocation-free ELL packer, through the C ABI.

It serves callers that cannot allocate device memory when they call in (another allocator
owns the GPU's memory, or the calling loop forbids allocation); its scratch is a fixed
array inside the library that every call on a device shares. This file is collected last,
so that a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1209_5421_gb300.meshes import p1_poisson

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    from paper_1209_5421_gb300 import amg, build

    build.build()
    return amg


def _pack(amg, fn, rowptr, col, val, width, diag_first):
    import torch

    rows = len(rowptr) - 1
    d = lambda a: torch.as_tensor(a).cuda()  # noqa: E731
    rp, cl, vl = d(rowptr), d(col), d(val)
    Aj = torch.full((rows * width,), 7, dtype=torch.int32, device="cuda")
    Ax = torch.full((rows * width,), 7.0, dtype=torch.float64, device="cuda")
    st = fn(rows, rp.data_ptr(), cl.data_ptr(), vl.data_ptr(), width, int(diag_first),
            Aj.data_ptr(), Ax.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, Aj.cpu().numpy(), Ax.cpu().numpy()


def test_matches_allocating_entry_point_on_consecutive_calls(lib):
    L = lib.lib()
    probs = [p1_poisson(33, jitter=0.2, seed=1), p1_poisson(70, jitter=0.1, graded=True, seed=2)]
    for prob, diag_first in ((probs[0], True), (probs[1], False), (probs[0], False)):
        width = int(np.diff(prob.rowptr).max())
        st0, Aj0, Ax0 = _pack(lib, L.amg_csr_to_ell, prob.rowptr, prob.col, prob.val, width,
                              diag_first)
        st1, Aj1, Ax1 = _pack(lib, L.amg_csr_to_ell_noalloc, prob.rowptr, prob.col, prob.val,
                              width, diag_first)
        assert st0 == lib.OK and st1 == lib.OK
        np.testing.assert_array_equal(Aj1, Aj0)  # integer / copied values: bit-exact
        np.testing.assert_array_equal(Ax1, Ax0)


def test_overflow_is_reported_and_does_not_stick(lib):
    L = lib.lib()
    prob = p1_poisson(17, jitter=0.2, seed=3)
    width = int(np.diff(prob.rowptr).max())
    st, _, _ = _pack(lib, L.amg_csr_to_ell_noalloc, prob.rowptr, prob.col, prob.val, width - 1, 1)
    assert st == lib.ERR_INVALID_ARG
    st, Aj, Ax = _pack(lib, L.amg_csr_to_ell_noalloc, prob.rowptr, prob.col, prob.val, width, 1)
    assert st == lib.OK
    st0, Aj0, Ax0 = _pack(lib, L.amg_csr_to_ell, prob.rowptr, prob.col, prob.val, width, 1)
    np.testing.assert_array_equal(Aj, Aj0)
    np.testing.assert_array_equal(Ax, Ax0)


def test_limits_and_host_arrays_rejected(lib):
    import torch

    L = lib.lib()
    tiny = torch.zeros(4, dtype=torch.int32, device="cuda")
    tinyd = torch.zeros(4, dtype=torch.float64, device="cuda")
    # more rows than the static scratch covers: rejected before any array is read
    st = L.amg_csr_to_ell_noalloc(4194305, tiny.data_ptr(), tiny.data_ptr(), tinyd.data_ptr(), 1,
                                  1, tiny.data_ptr(), tinyd.data_ptr(), None)
    assert st == lib.ERR_UNSUPPORTED
    prob = p1_poisson(9)
    Aj = np.empty(prob.n * 5, np.int32)
    Ax = np.empty(prob.n * 5)
    st = L.amg_csr_to_ell_noalloc(prob.n, prob.rowptr.ctypes.data, prob.col.ctypes.data,
                                  prob.val.ctypes.data, 5, 1, Aj.ctypes.data, Ax.ctypes.data, None)
    assert st == lib.ERR_INVALID_ARG


def _golden_ell():
    import os

    d = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "ell_example.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        d[k] = [float(t) for t in v]
    return d


def test_paper_worked_example(lib):
    # the ELL example printed with the packing (3 x 4 matrix, K = 3, column-major Aj / Ax)
    L = lib.lib()
    g = _golden_ell()
    rp = np.array(g["rowptr"], np.int32)
    cl = np.array(g["col"], np.int32)
    vl = np.array(g["val"])
    width = int(g["width"][0])
    for _ in range(2):  # two calls in a row: the shared scratch carries nothing over
        st, Aj, Ax = _pack(lib, L.amg_csr_to_ell_noalloc, rp, cl, vl, width, False)
        assert st == lib.OK
        np.testing.assert_array_equal(Aj, np.array(g["Aj"], np.int32))
        np.testing.assert_array_equal(Ax, np.array(g["Ax"]))


def test_overflow_in_a_late_block_only(lib):
    # more than one 256-row block, and only a row of the last block is too long: the count of
    # that block must reach the total (every block's count is summed)
    L = lib.lib()
    prob = p1_poisson(40, jitter=0.2, seed=4)  # 38^2 = 1444 rows: 6 blocks
    assert prob.n > 5 * 256
    deg = np.diff(prob.rowptr)
    width = int(deg.max())
    # a matrix whose only rows of `width` entries lie in the last block: drop the last entry
    # of every such row before it
    cut = 5 * 256
    short = np.zeros(prob.n, bool)
    short[:cut] = deg[:cut] == width
    keep = np.ones(len(prob.col), bool)
    keep[prob.rowptr[1:][short] - 1] = False
    rowptr = np.concatenate([[0], np.cumsum(deg - short)]).astype(np.int32)
    col, val = prob.col[keep], prob.val[keep]
    d2 = np.diff(rowptr)
    assert d2[:cut].max() < width and d2[cut:].max() == width
    st, _, _ = _pack(lib, L.amg_csr_to_ell_noalloc, rowptr, col, val, width - 1, 1)
    assert st == lib.ERR_INVALID_ARG
    assert b"width" in L.amg_last_error()
    st, Aj, Ax = _pack(lib, L.amg_csr_to_ell_noalloc, rowptr, col, val, width, 1)
    assert st == lib.OK
    st0, Aj0, Ax0 = _pack(lib, L.amg_csr_to_ell, rowptr, col, val, width, 1)
    assert st0 == lib.OK
    np.testing.assert_array_equal(Aj, Aj0)
    np.testing.assert_array_equal(Ax, Ax0)


def test_failures_set_the_error_text(lib):
    import torch

    L = lib.lib()
    tiny = torch.zeros(4, dtype=torch.int32, device="cuda")
    tinyd = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = L.amg_csr_to_ell_noalloc(4194305, tiny.data_ptr(), tiny.data_ptr(), tinyd.data_ptr(), 1,
                                  1, tiny.data_ptr(), tinyd.data_ptr(), None)
    assert st == lib.ERR_UNSUPPORTED and b"4,194,304" in L.amg_last_error()
    prob = p1_poisson(9)
    Aj = np.empty(prob.n * 5, np.int32)
    Ax = np.empty(prob.n * 5)
    st = L.amg_csr_to_ell_noalloc(prob.n, prob.rowptr.ctypes.data, prob.col.ctypes.data,
                                  prob.val.ctypes.data, 5, 1, Aj.ctypes.data, Ax.ctypes.data, None)
    assert st == lib.ERR_INVALID_ARG and b"device arrays" in L.amg_last_error()


def test_capturing_stream_is_refused_and_the_capture_goes_on(lib):
    # the call reads its result back and waits on its stream, which a capturing stream does
    # not allow: it must refuse before any work and leave the caller's capture intact
    import torch

    L = lib.lib()
    prob = p1_poisson(17, jitter=0.2, seed=3)
    width = int(np.diff(prob.rowptr).max())
    st, _, _ = _pack(lib, L.amg_csr_to_ell_noalloc, prob.rowptr, prob.col, prob.val, width, 1)
    assert st == lib.OK  # the first call on the device (scratch address) outside any capture
    d = lambda a: torch.as_tensor(a).cuda()  # noqa: E731
    rp, cl, vl = d(prob.rowptr), d(prob.col), d(prob.val)
    Aj = torch.full((prob.n * width,), 7, dtype=torch.int32, device="cuda")
    Ax = torch.full((prob.n * width,), 7.0, dtype=torch.float64, device="cuda")
    a = torch.arange(1000, dtype=torch.float64, device="cuda")
    out = torch.zeros_like(a)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        s = torch.cuda.current_stream()
        st = L.amg_csr_to_ell_noalloc(prob.n, rp.data_ptr(), cl.data_ptr(), vl.data_ptr(), width,
                                      1, Aj.data_ptr(), Ax.data_ptr(),
                                      ctypes.c_void_p(s.cuda_stream))
        out.copy_(a * 3.0)
    assert st == lib.ERR_UNSUPPORTED and b"capturing" in L.amg_last_error()
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), 3.0 * np.arange(1000))
    assert (Aj.cpu().numpy() == 7).all() and (Ax.cpu().numpy() == 7.0).all()  # no work done
    st, Aj1, Ax1 = _pack(lib, L.amg_csr_to_ell_noalloc, prob.rowptr, prob.col, prob.val, width, 1)
    st0, Aj0, Ax0 = _pack(lib, L.amg_csr_to_ell, prob.rowptr, prob.col, prob.val, width, 1)
    assert st == lib.OK and st0 == lib.OK
    np.testing.assert_array_equal(Aj1, Aj0)
    np.testing.assert_array_equal(Ax1, Ax0)
