"""GPU: failure detection, with faults made on the host or by a bounded wait that runs out.

No test here makes the GPU fault, trap or hang:
* barrier timeouts: a host-set fault (amg_debug_barrier_fault) shortens the wait limit of the
  cycle kernel's grid barrier to 1 ms and makes its first barrier wait for one arrival more
  than the grid makes, so the wait runs out; the solve must return AMG_ERR_TIMEOUT and the
  next solve on the same hierarchy must be correct. The same for the team barrier of batches;
* allocation failures: a host-set fault (amg_debug_fail_allocation) fails the k-th device
  allocation; the call must return AMG_ERR_OOM and release everything it had allocated
  (the default memory pool's bytes in use are the same before and after).
"""
import numpy as np
import pytest

from paper_1209_5421_gb300.meshes import p1_poisson

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amg():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    from paper_1209_5421_gb300 import amg as A
    from paper_1209_5421_gb300 import build

    build.build()
    yield A
    A.debug_fail_allocation(0)


def _true_rel(prob, x):
    A = prob.to_scipy()
    return np.linalg.norm(prob.b - A @ x) / np.linalg.norm(prob.b)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cycle_barrier_timeout_then_recovery(amg, prec):
    # 9,025 unknowns: the finest level runs grid-wide, so the cycle kernel meets grid barriers
    prob = p1_poisson(97, jitter=0.2, seed=1, rhs="normal")
    kw = dict(cycle_prec=amg.FP32, outer=amg.OUTER_FGMRES) if prec == "fp32" else {}
    H = amg.Hierarchy.from_problem(prob, **kw)
    x0, it0, _, st0 = H.solve(prob.b, 1e-8)
    assert st0 == amg.OK
    H.debug_barrier_fault(limit_ns=1_000_000, extra=1)
    with pytest.raises(amg.AmgError) as ei:
        H.solve(prob.b, 1e-8)
    assert ei.value.status == amg.ERR_TIMEOUT
    # the fault off again: the same hierarchy solves as before, bit for bit
    H.debug_barrier_fault(0, 0)
    x1, it1, _, st1 = H.solve(prob.b, 1e-8)
    assert st1 == amg.OK and it1 == it0
    assert np.array_equal(x1, x0)
    assert _true_rel(prob, x1) <= 1e-8
    H.close()


def test_short_limit_alone_does_not_fire(amg):
    # a 1 ms limit with every CTA arriving: no barrier of this solve waits that long
    prob = p1_poisson(97, jitter=0.2, seed=2, rhs="normal")
    H = amg.Hierarchy.from_problem(prob)
    H.debug_barrier_fault(limit_ns=1_000_000, extra=0)
    x, it, rr, st = H.solve(prob.b, 1e-8)
    assert st == amg.OK and _true_rel(prob, x) <= 1e-8
    H.close()


def test_team_barrier_timeout_then_recovery(amg):
    # the largest system forms a team of CTAs; its first team barrier is made to run out
    probs = [p1_poisson(n, jitter=0.2, seed=3 + k, rhs="normal")
             for k, n in enumerate((17, 45, 65, 257))]
    B = amg.Batch.from_problems(probs, cycle_prec=amg.FP32)
    rhs = np.concatenate([p.b for p in probs])
    x0, it0, _, st0 = B.solve(rhs, 1e-8)
    assert (st0 == amg.OK).all()
    team = B.teams()
    assert team.max() > 1
    B.debug_barrier_fault(limit_ns=1_000_000, extra=1)
    _, _, _, st = B.solve(rhs, 1e-8)
    for k in range(len(probs)):
        if team[k] > 1:
            assert st[k] == amg.ERR_TIMEOUT, (k, st)
        else:
            assert st[k] == amg.OK, (k, st)  # one-CTA systems wait on no team barrier
    B.debug_barrier_fault(0, 0)
    x1, it1, _, st1 = B.solve(rhs, 1e-8)
    assert (st1 == amg.OK).all() and np.array_equal(it1, it0)
    assert np.array_equal(x1, x0)
    B.close()


def _setup_and_solve(amg, prob, **kw):
    H = amg.Hierarchy.from_problem(prob, **kw)
    try:
        x, it, rr, st = H.solve(prob.b, 1e-8, check=True)
    finally:
        H.close()
    return x, it


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_allocation_failures_release_everything(amg, prec):
    import torch

    prob = p1_poisson(97, jitter=0.2, seed=4, rhs="normal")
    kw = dict(cycle_prec=amg.FP32, outer=amg.OUTER_FGMRES) if prec == "fp32" else {}
    xr, itr = _setup_and_solve(amg, prob, **kw)  # warm (pool, kernels) and the reference
    torch.cuda.synchronize()
    base = amg.pool_bytes_in_use(torch.cuda.current_device())
    failed = 0
    for k in range(1, 400):
        amg.debug_fail_allocation(k)
        try:
            x, it = _setup_and_solve(amg, prob, **kw)
        except amg.AmgError as e:
            assert e.status == amg.ERR_OOM, e
            failed += 1
            ok = False
        else:
            ok = True
        finally:
            amg.debug_fail_allocation(0)
        torch.cuda.synchronize()
        assert amg.pool_bytes_in_use(torch.cuda.current_device()) == base, k
        if ok:  # k is past the last allocation of setup + solve: nothing failed
            assert it == itr and np.array_equal(x, xr)
            break
    assert failed >= 10  # setup and the first solve allocate many buffers; each was tried


def test_failed_lazy_allocation_leaves_the_hierarchy_usable(amg):
    # the FP32 cycle's buffers are allocated on the first solve: fail one of them, then solve
    # again on the same hierarchy
    prob = p1_poisson(97, jitter=0.2, seed=5, rhs="normal")
    xr, itr = _setup_and_solve(amg, prob, cycle_prec=amg.FP32, outer=amg.OUTER_FGMRES)
    H = amg.Hierarchy.from_problem(prob, cycle_prec=amg.FP32, outer=amg.OUTER_FGMRES)
    for k in (1, 3, 7):
        amg.debug_fail_allocation(k)
        try:
            with pytest.raises(amg.AmgError) as ei:
                H.solve(prob.b, 1e-8)
            assert ei.value.status == amg.ERR_OOM
        finally:
            amg.debug_fail_allocation(0)
    x, it, rr, st = H.solve(prob.b, 1e-8)
    assert st == amg.OK and it == itr and np.array_equal(x, xr)
    H.close()


def test_batch_setup_allocation_failure(amg):
    import torch

    probs = [p1_poisson(n, jitter=0.2, seed=6 + k, rhs="normal") for k, n in enumerate((17, 33))]
    B = amg.Batch.from_problems(probs, cycle_prec=amg.FP32)
    B.close()
    torch.cuda.synchronize()
    base = amg.pool_bytes_in_use(torch.cuda.current_device())
    for k in (1, 5, 20, 60):
        amg.debug_fail_allocation(k)
        try:
            B = amg.Batch.from_problems(probs, cycle_prec=amg.FP32)
        except amg.AmgError as e:
            assert e.status == amg.ERR_OOM
        else:
            B.close()
        finally:
            amg.debug_fail_allocation(0)
        torch.cuda.synchronize()
        assert amg.pool_bytes_in_use(torch.cuda.current_device()) == base, k
