"""GPU: the continuous-batching server (resident hierarchies, HBM-budget admission).

Each request's result must be the same alone and in the mix: bitwise, because every system is
computed by one CTA of fixed size (batch lane) or by the deterministic single-system kernel
(large lane), whatever else is in flight. Results are also checked against the FP64 residual
and the oracle, and the resident device bytes never exceed the budget.
"""
import time

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
    return A


SIZES = [33, 65, 17, 129, 97, 45, 257]  # 257 x 257 nodes: the large lane below


def _problems():
    return {f"m{k}": p1_poisson(n, jitter=0.2, seed=10 + k, rhs="normal", graded=(k == 4),
                                kappa_blocks=16 if k == 4 else 0)
            for k, n in enumerate(SIZES)}


def _requests(probs, count, seed):
    rng = np.random.default_rng(seed)
    keys = list(probs)
    out = []
    for i in range(count):
        key = keys[rng.integers(len(keys))]
        out.append((key, rng.standard_normal(probs[key].n)))
    return out


def _solo(amg, prob, b, large):
    """The same request alone, by the same lane's code."""
    from paper_1209_5421_gb300.serve import Server

    S = Server(workers=1, large_unknowns=large)
    S.register("k", prob.rowptr, prob.col, prob.val, prob.x, prob.y)
    r = S.submit("k", b)
    S.drain()
    S.close()
    return r


def test_results_same_alone_and_in_the_mix(amg, oracle_mod):
    from paper_1209_5421_gb300.serve import Server

    probs = _problems()
    large = 40_000  # the 257 x 257 system (65k unknowns) takes the large lane
    reqs = _requests(probs, 40, seed=3)
    S = Server(workers=4, large_unknowns=large)
    for k, p in probs.items():
        S.register(k, p.rowptr, p.col, p.val, p.x, p.y)
    rng = np.random.default_rng(5)
    handles = []
    for key, b in reqs:  # arrivals spread over time, while earlier ones run
        handles.append(S.submit(key, b))
        time.sleep(float(rng.exponential(0.002)))
    S.drain()
    st = S.stats()
    S.close()
    assert st["completed"] == len(reqs), st
    assert st["large_lane"] > 0 and st["batches"] > 1
    checked = set()
    for r, (key, b) in zip(handles, reqs):
        p = probs[key]
        assert r.status == amg.OK, (key, r.status)
        A = p.to_scipy()
        assert np.linalg.norm(b - A @ r.x) / np.linalg.norm(b) <= 1e-8
        if key in checked:
            continue
        checked.add(key)
        alone = _solo(amg, p, b, large)
        assert alone.lane == r.lane
        assert np.array_equal(alone.x, r.x), key
        assert alone.iters == r.iters
        if p.n < 20_000:  # the oracle on the small systems
            O = oracle_mod.Hierarchy.from_problem(p)
            xo, _, _, _ = O.solve(b, 1e-8)
            assert np.linalg.norm(r.x - xo) / np.linalg.norm(xo) <= 1e-6


def test_budget_admission_and_eviction(amg):
    from paper_1209_5421_gb300.serve import Server, setup_estimate

    probs = _problems()
    del probs["m6"]
    # room for the largest hierarchy (its real bytes, or the estimate it is admitted by, if
    # larger) and a bit more: the others must take turns
    big = max(probs.values(), key=lambda p: p.n)
    h = amg.Hierarchy.from_problem(big, cycle_prec=amg.FP32)
    amg.Batch.over([h], threads=1024).close()
    base = max(h.nbytes, setup_estimate(big.n, len(big.col)))
    budget = int(1.3 * base)
    h.close()
    total = base * sum(p.n for p in probs.values()) / big.n
    assert total > 1.5 * budget  # the mix does not fit at once
    S = Server(budget_bytes=budget, workers=2)
    for k, p in probs.items():
        S.register(k, p.rowptr, p.col, p.val, p.x, p.y)
    reqs = _requests(probs, 24, seed=7)
    handles = [S.submit(k, b) for k, b in reqs]
    S.drain()
    st = S.stats()
    S.close()
    assert st["completed"] == len(reqs), st
    assert st["evictions"] > 0
    # the peak: within the budget, plus the outer directions that solves added on demand
    # (the graded system's batched solves need more than the 32 allocated at first)
    assert st["max_resident_bytes"] <= budget + st["grown_bytes"], st
    for r, (key, b) in zip(handles, reqs):
        A = probs[key].to_scipy()
        assert r.status == amg.OK
        assert np.linalg.norm(b - A @ r.x) / np.linalg.norm(b) <= 1e-8


def test_waiting_matrices_set_up_together(amg):
    # new batch-lane matrices queued at the same time are set up by one amg_setup_many: each
    # result is still the one a request alone gets (bitwise), and the charged bytes are the
    # resident hierarchies' own
    from paper_1209_5421_gb300.serve import Server

    probs = _problems()
    del probs["m6"]
    large = 40_000
    S = Server(workers=2, large_unknowns=large)
    for k, p in probs.items():
        S.register(k, p.rowptr, p.col, p.val, p.x, p.y)
    rng = np.random.default_rng(9)
    with S.cv:  # all queued before the setup thread looks
        reqs = [(k, rng.standard_normal(p.n)) for k, p in probs.items()]
        handles = [S.submit(k, b) for k, b in reqs]
    S.drain()
    st = S.stats()
    assert S.used == sum(e.nbytes for e in S.res.values()) == sum(e.h.nbytes for e in S.res.values())
    S.close()
    assert st["group_setups"] == 1 and st["setups"] == len(probs), st
    for r, (key, b) in zip(handles, reqs):
        assert r.status == amg.OK and r.lane == "batch", (key, r.status, r.lane)
        alone = _solo(amg, probs[key], b, large)
        assert np.array_equal(alone.x, r.x) and alone.iters == r.iters, key
