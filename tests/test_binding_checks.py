"""The Python binding checks what a raw pointer cannot carry: lengths and element types.

The C ABI takes plain pointers, so a buffer shorter than the count the call reads, or a tensor
whose bytes are not the type the call reads (int64 row pointers, float32 values), would be
read past its end or misread. The binding rejects both before calling the library. Runs
without a GPU: every rejected call raises before the library is reached, and the accepted
ones reach it (and fail there with a CUDA status, as nothing runs without a GPU).
"""
import numpy as np
import pytest
import torch

from paper_1209_5421_gb300 import amg, build
from paper_1209_5421_gb300.meshes import p1_poisson


@pytest.fixture(scope="module")
def prob():
    build.build()
    return p1_poisson(9, jitter=0.2, seed=0, rhs="normal")


def _args(p):
    return [p.rowptr, p.col, p.val, p.x, p.y]


@pytest.mark.parametrize("k,bad", [(2, lambda a: a[:-1]), (3, lambda a: a[:-1]),
                                   (4, lambda a: np.append(a, 0.0))])
def test_setup_rejects_wrong_lengths(prob, k, bad):
    args = _args(prob)
    args[k] = bad(args[k])
    with pytest.raises(ValueError):
        amg.Hierarchy(*args)
    with pytest.raises(ValueError):
        amg.Hierarchy(*_args(prob), z=np.zeros(prob.n + 1))
    with pytest.raises(ValueError):
        amg.Hierarchy(np.zeros(0, np.int32), prob.col, prob.val, prob.x, prob.y)


@pytest.mark.parametrize("k,dtype", [(0, torch.int64), (1, torch.int64), (2, torch.float32),
                                     (3, torch.float32)])
def test_setup_rejects_tensors_of_another_type(prob, k, dtype):
    args = [torch.as_tensor(a) for a in _args(prob)]
    args[k] = args[k].to(dtype)
    with pytest.raises(TypeError):
        amg.Hierarchy(*args)


def test_correct_inputs_reach_the_library(prob):
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the setup would run on it")
    for args in (_args(prob), [torch.as_tensor(a) for a in _args(prob)],
                 [a.astype(np.int64) if a.dtype == np.int32 else a for a in _args(prob)]):
        with pytest.raises(amg.AmgError) as e:  # numpy int64 is converted, not rejected
            amg.Hierarchy(*args)
        assert e.value.status == amg.ERR_CUDA


def _unbuilt(n, level_n=None):
    """A Hierarchy object with no library state, for checks made before any C call."""
    h = amg.Hierarchy.__new__(amg.Hierarchy)
    h.h, h.n = None, n
    if level_n is not None:
        h.level_info = lambda l: {"n": level_n}
    return h


def test_solve_checks_b_and_x(prob):
    h = _unbuilt(prob.n)
    with pytest.raises(ValueError):
        h.solve(prob.b[:-1])
    with pytest.raises(TypeError):
        h.solve(torch.as_tensor(prob.b).float())
    with pytest.raises(TypeError):
        h.solve(prob.b, x=np.empty(prob.n, np.float32))
    with pytest.raises(ValueError):
        h.solve(prob.b, x=np.empty(prob.n - 1))
    with pytest.raises(ValueError):
        h.solve(torch.as_tensor(prob.b), x=torch.empty(prob.n + 1, dtype=torch.float64))


def test_cycle_and_smoother_check_lengths():
    h = _unbuilt(100, level_n=25)
    with pytest.raises(ValueError):
        h.apply_cycle(1, np.zeros(24))
    with pytest.raises(ValueError):
        h.smooth(1, np.zeros(25), np.zeros(26))
    with pytest.raises(TypeError):
        h.smooth(1, torch.zeros(25, dtype=torch.float32), np.zeros(25))


def test_batch_checks_lengths(prob):
    h = amg.Batch.__new__(amg.Batch)
    h.b, h.n, h.nprob = None, 2 * prob.n, 2
    with pytest.raises(ValueError):
        h.solve(np.zeros(2 * prob.n - 1))
    with pytest.raises(TypeError):
        h.solve(np.zeros(2 * prob.n), x=np.zeros(2 * prob.n, np.float32))
    bad = (prob.rowptr, prob.col, prob.val, prob.x[:-1], prob.y)
    with pytest.raises(ValueError):
        amg.Batch([(prob.rowptr, prob.col, prob.val, prob.x, prob.y), bad])


def test_ell_packer_checks_rowptr(prob):
    rp = prob.rowptr.copy()
    with pytest.raises(ValueError):  # points past the end of col
        amg.csr_to_ell(np.append(rp[:-1], rp[-1] + 5), prob.col, prob.val, 9)
    rp2 = rp.copy()
    rp2[3], rp2[4] = rp2[4], rp2[3]
    with pytest.raises(ValueError):  # not non-decreasing
        amg.csr_to_ell(rp2, prob.col, prob.val, 9)
    with pytest.raises(ValueError):
        amg.csr_to_ell(rp, prob.col, prob.val[:-1], 9)


def test_concatenate_lays_out_the_block_diagonal_matrix():
    # amg.concatenate (the layout amg_batch_setup and amg_setup_many take): global row
    # pointers and columns of the block-diagonal matrix, coordinates end to end, row offsets
    import scipy.sparse as sp

    probs = [p1_poisson(n, jitter=0.2, seed=n, rhs="normal") for n in (5, 9, 4, 12)]
    ro, rp, cl, vl, xx, yy = amg.concatenate([(p.rowptr, p.col, p.val, p.x, p.y) for p in probs])
    assert rp.dtype == np.int32 and cl.dtype == np.int32 and vl.dtype == np.float64
    np.testing.assert_array_equal(ro, np.cumsum([0] + [p.n for p in probs]))
    A = sp.csr_matrix((vl, cl, rp), shape=(ro[-1], ro[-1]))
    B = sp.block_diag([p.to_scipy() for p in probs], format="csr")
    assert abs(A - B).max() == 0.0 and A.nnz == B.nnz
    np.testing.assert_array_equal(xx, np.concatenate([p.x for p in probs]))
    np.testing.assert_array_equal(yy, np.concatenate([p.y for p in probs]))
    bad = [(p.rowptr, p.col, p.val, p.x, p.y) for p in probs]
    bad[2] = (probs[2].rowptr, probs[2].col, probs[2].val[:-1], probs[2].x, probs[2].y)
    with pytest.raises(ValueError):
        amg.concatenate(bad)


def test_setup_many_rejects_unknown_options(prob):
    with pytest.raises(TypeError):
        amg.setup_many([_args(prob)], outer_method=1)
