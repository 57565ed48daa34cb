"""The serving loop's host logic on the CPU, with the GPU work replaced by fakes.

The real `Server` runs (its setup thread, batch workers and large-lane thread, admission,
eviction and queues); only the hierarchy and batch objects are stand-ins that solve exactly
with scipy, report a device size, and record when they run. This checks the scheduling
invariants without a GPU:
  * every request gets the solution of its own system, through the lane its size selects;
  * admission: with the setup estimate above the real size the resident bytes never exceed
    the budget and idle hierarchies are evicted least recently used first; real sizes above
    the estimate, and growth during solves, are charged and evicted back under the budget;
    a matrix larger than the whole budget fails its own requests;
  * continuous batching: a request that arrives while a batch runs starts beside it on a free
    worker (with one worker it can only follow);
  * a large-lane solve never overlaps a batch solve or a setup, whichever comes first (it has
    the GPU to itself);
  * a request the server cannot set up (unknown key, rejected or oversized matrix) ends alone
    with a status, and the others are served.
The same server on the GPU is tested in test_gpu_serve.py.
"""
import contextlib
import importlib.util
import os
import sys
import threading
import time

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_1209_5421_gb300 import amg
from paper_1209_5421_gb300.meshes import p1_poisson

BYTES_PER_UNKNOWN = 1000  # the fakes' device size (below the server's setup estimate)
# a copy of serve.py to test instead of the package's (test_serve_mutants.py plants mistakes)
SERVE_UNDER_TEST = "AMG_SERVE_UNDER_TEST"


def serve_module():
    path = os.environ.get(SERVE_UNDER_TEST)
    if not path:
        from paper_1209_5421_gb300 import serve
        return serve
    spec = importlib.util.spec_from_file_location("paper_1209_5421_gb300._serve_under_test", path)
    mod = importlib.util.module_from_spec(spec)
    mod.__package__ = "paper_1209_5421_gb300"  # its relative imports: the package's modules
    sys.modules[spec.name] = mod  # dataclasses look their module up there
    spec.loader.exec_module(mod)
    return mod


class Log:
    def __init__(self):
        self.lock = threading.Lock()
        self.intervals = []  # (kind, t0, t1)
        self.closed = []     # sizes of closed hierarchies, in order
        self.groups = []     # sizes of the multi-system setups (amg.setup_many calls)
        self.running = {}    # kind -> spans in progress

    @contextlib.contextmanager
    def span(self, kind, hold=0.003):
        t0 = time.perf_counter()
        with self.lock:
            self.running[kind] = self.running.get(kind, 0) + 1
        time.sleep(hold)  # long enough for overlaps to show
        yield
        with self.lock:
            self.running[kind] -= 1
            self.intervals.append((kind, t0, time.perf_counter()))


def _solve(rowptr, col, val, b):
    n = len(rowptr) - 1
    return spla.spsolve(sp.csr_matrix((val, col, rowptr), shape=(n, n)).tocsc(), b)


def make_fakes(torch, log, bytes_per_unknown=BYTES_PER_UNKNOWN, grow_per_solve=0,
               batch_hold=0.003, large_hold=0.003):
    class FakeHierarchy:
        def __init__(self, rowptr, col, val, x, y, z=None, cycle_prec=None, outer=None):
            if np.asarray(val)[0] <= 0:  # as the library's check of the diagonal
                raise amg.AmgError(amg.ERR_BAD_MATRIX, "amg_setup: stand-in rejects the matrix")
            with log.span("setup"):
                self.A = (np.asarray(rowptr), np.asarray(col), np.asarray(val))
                self.n = len(rowptr) - 1
                self.nbytes = bytes_per_unknown * self.n

        def solve(self, b, tol, stream=None):
            with log.span("large", hold=large_hold):
                x = _solve(*self.A, b.numpy())
            self.nbytes += grow_per_solve  # as the outer iteration's directions are allocated
            return torch.from_numpy(x), 1, 0.0, amg.OK

        def close(self):
            with log.lock:
                log.closed.append(self.n)

    class FakeBatch:
        def __init__(self, hs):
            self.hs = hs
            self.row_off = np.zeros(len(hs) + 1, np.int64)
            self.row_off[1:] = np.cumsum([h.n for h in hs])

        @classmethod
        def over(cls, hierarchies, threads=0, stream=None):
            # a system's batched workspace belongs to its hierarchy: one system, one slot
            assert len({id(h) for h in hierarchies}) == len(hierarchies), "a system twice"
            return cls(list(hierarchies))

        def solve(self, rhs, tol, stream=None):
            with log.span("batch", hold=batch_hold):
                r = rhs.numpy()
                x = np.concatenate([_solve(*h.A, r[self.row_off[k]:self.row_off[k + 1]])
                                    for k, h in enumerate(self.hs)])
            for h in self.hs:
                h.nbytes += grow_per_solve
            k = len(self.hs)
            return torch.from_numpy(x), np.ones(k, int), np.zeros(k), np.zeros(k, int)

        def close(self):
            pass

    return FakeHierarchy, FakeBatch


@pytest.fixture
def server_cls(monkeypatch):
    import torch

    monkeypatch.setattr(torch.cuda, "set_device", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    Server = serve_module().Server

    log = Log()
    made = []

    def make(bytes_per_unknown=BYTES_PER_UNKNOWN, grow_per_solve=0, batch_hold=0.003,
             large_hold=0.003, **kw):
        H, B = make_fakes(torch, log, bytes_per_unknown, grow_per_solve, batch_hold, large_hold)

        def setup_many(problems, cycle_prec=None, outer=None):
            # as amg_setup_many: one hierarchy per system, or the first rejection for all
            with log.lock:
                log.groups.append(len(problems))
            return [H(*p, cycle_prec=cycle_prec, outer=outer) for p in problems]

        monkeypatch.setattr(amg, "Hierarchy", H)
        monkeypatch.setattr(amg, "Batch", B)
        monkeypatch.setattr(amg, "setup_many", setup_many)
        S = Server(**kw)
        S.dev = torch.device("cpu")  # before the first request: the fakes run on the host
        made.append(S)
        return S

    yield make, log
    for S in made:  # also when the test failed: no server thread outlives its test
        S.close()


def _consistent(S):
    """The charged bytes are the resident hierarchies' current bytes."""
    ents = list(S.res.values())
    return S.used == sum(e.h.nbytes for e in ents) == sum(e.nbytes for e in ents)


def _problems(sizes):
    return {f"m{k}": p1_poisson(n, jitter=0.2, seed=20 + k, rhs="normal")
            for k, n in enumerate(sizes)}


def _register(S, probs):
    for key, p in probs.items():
        S.register(key, p.rowptr, p.col, p.val, p.x, p.y)


def _overlaps(log, a, b):
    A = [(t0, t1) for k, t0, t1 in log.intervals if k == a]
    B = [(t0, t1) for k, t0, t1 in log.intervals if k == b]
    return [(x, y) for x in A for y in B if x[0] < y[1] and y[0] < x[1]]


def test_results_lanes_and_exclusive_large_lane(server_cls):
    make, log = server_cls
    probs = _problems([9, 17, 12, 33, 14, 29])  # 49 .. 961 unknowns
    large = 500  # the 33 x 33 and 29 x 29 node systems take the large lane
    S = make(workers=3, large_unknowns=large)
    _register(S, probs)
    rng = np.random.default_rng(5)
    reqs = []
    for i in range(40):
        key = f"m{rng.integers(len(probs))}"
        reqs.append((key, S.submit(key, rng.standard_normal(probs[key].n))))
        if i % 7 == 0:
            time.sleep(0.002)
    S.drain(timeout=120)
    st = S.stats()
    S.close()
    assert st["completed"] == len(reqs)
    assert st["setups"] == len({k for k, _ in reqs}) and st["evictions"] == 0
    for key, r in reqs:
        p = probs[key]
        assert r.done.is_set() and r.status == amg.OK
        assert r.lane == ("large" if p.n > large else "batch"), (key, r.lane)
        np.testing.assert_allclose(r.x, _solve(p.rowptr, p.col, p.val, r.b), rtol=0, atol=1e-12)
    assert any(k == "large" for k, _, _ in log.intervals)
    assert not _overlaps(log, "large", "batch")
    assert not _overlaps(log, "large", "setup")


@pytest.mark.parametrize("workers", [1, 2])
def test_arrivals_during_a_batch_start_beside_it(server_cls, workers):
    """Continuous batching: a request that becomes ready while a batch is on the GPU starts in
    a launch of its own on a free worker, overlapping the running one, instead of waiting for
    it. With one worker (the control) the second batch can only follow the first."""
    make, log = server_cls
    probs = _problems([9, 12])
    S = make(workers=workers, batch_hold=0.3, large_unknowns=10 ** 6)
    _register(S, probs)
    r0 = S.submit("m0", np.ones(probs["m0"].n))
    t0 = time.perf_counter()
    while not log.running.get("batch") and time.perf_counter() - t0 < 30:
        time.sleep(0.002)  # until m0's batch is on the (stand-in) GPU
    assert log.running.get("batch") == 1
    r1 = S.submit("m1", np.ones(probs["m1"].n))
    S.drain(timeout=60)
    S.close()
    assert r0.status == r1.status == amg.OK and r0.lane == r1.lane == "batch"
    batches = [(t0, t1) for k, t0, t1 in log.intervals if k == "batch"]
    assert len(batches) == 2
    overlap = _overlaps(log, "batch", "batch")
    overlapping = [(a, b) for a, b in overlap if a != b]
    assert bool(overlapping) == (workers > 1), batches


def _wait_running(log, kind):
    t0 = time.perf_counter()
    while not log.running.get(kind) and time.perf_counter() - t0 < 30:
        time.sleep(0.002)
    assert log.running.get(kind) == 1, kind


@pytest.mark.parametrize("first", ["batch", "large"])
def test_large_lane_has_the_gpu_to_itself(server_cls, first):
    """A large-lane request that arrives while a batch runs waits for it to finish; while a
    large solve runs, neither a batch of a resident matrix nor a new matrix's setup starts:
    the large solve never overlaps either."""
    make, log = server_cls
    probs = _problems([9, 14, 10])  # 49 and 64 unknowns: batch lane; 144: large lane
    S = make(workers=2, large_unknowns=100, batch_hold=0.25, large_hold=0.25)
    _register(S, probs)
    ones = {k: np.ones(p.n) for k, p in probs.items()}
    if first == "batch":
        reqs = [S.submit("m0", ones["m0"])]
        _wait_running(log, "batch")
        reqs.append(S.submit("m1", ones["m1"]))  # large, while the batch runs
    else:
        reqs = [S.submit("m0", ones["m0"])]
        S.drain(timeout=60)  # m0 resident: its next request could start at once
        reqs.append(S.submit("m1", ones["m1"]))
        _wait_running(log, "large")
        reqs += [S.submit("m0", ones["m0"]), S.submit("m2", ones["m2"])]  # batch; new setup
    S.drain(timeout=60)
    S.close()
    assert all(r.status == amg.OK for r in reqs)
    assert {r.lane for r in reqs} == {"batch", "large"}
    assert not _overlaps(log, "large", "batch")
    assert not _overlaps(log, "large", "setup")


def test_budget_admission_lru_eviction(server_cls):
    setup_estimate = serve_module().setup_estimate

    make, log = server_cls
    probs = {f"m{k}": p1_poisson(n, jitter=0.2, seed=40 + k, rhs="normal")
             for k, n in enumerate([20, 21, 22, 21])}  # 324 .. 400 unknowns
    real = {k: BYTES_PER_UNKNOWN * p.n for k, p in probs.items()}
    est = {k: setup_estimate(p.n, len(p.col)) for k, p in probs.items()}
    assert all(est[k] > real[k] for k in probs)  # the estimate is an upper bound here
    # any two residents leave room for a setup's estimate, no three do
    budget = 2 * max(real.values()) + max(est.values())
    assert 3 * min(real.values()) + min(est.values()) > budget
    S = make(workers=2, budget_bytes=budget, large_unknowns=10 ** 6)
    _register(S, probs)
    for key in ["m0", "m1", "m0", "m2", "m3", "m1"]:  # one at a time: LRU = submission order
        r = S.submit(key, np.ones(probs[key].n))
        S.drain(timeout=60)
        assert r.status == amg.OK
        assert _consistent(S) and S.used <= budget
    st = S.stats()
    S.close()
    assert st["max_resident_bytes"] <= budget
    # m3 needs room with m1, m0, m2 resident: m1 goes (m0 was used after it); then m1 needs
    # room with m0, m2, m3 resident: m0 goes
    assert st["evictions"] == 2 and log.closed[:2] == [probs["m1"].n, probs["m0"].n]
    assert st["setups"] == 5


def test_real_size_above_the_estimate_is_evicted_back_under_the_budget(server_cls):
    setup_estimate = serve_module().setup_estimate

    make, _ = server_cls
    probs = _problems([20, 21, 22, 23])
    bpu = 3000  # real bytes per unknown, above the estimate
    assert all(setup_estimate(p.n, len(p.col)) < bpu * p.n for p in probs.values())
    # m3's estimate fits beside m2 but its real size does not: the server must evict m2 (idle)
    # after m3's setup
    budget = bpu * (probs["m2"].n + probs["m3"].n) - 1
    assert bpu * probs["m2"].n + setup_estimate(probs["m3"].n, len(probs["m3"].col)) <= budget
    S = make(bytes_per_unknown=bpu, workers=2, budget_bytes=budget, large_unknowns=10 ** 6)
    _register(S, probs)
    for key in ["m0", "m1", "m2", "m3", "m0"]:
        r = S.submit(key, np.ones(probs[key].n))
        S.drain(timeout=60)
        assert r.status == amg.OK
        assert key in S.res  # the hierarchy just set up stays
        assert _consistent(S) and S.used <= budget
    st = S.stats()
    S.close()
    assert st["evictions"] >= 3  # m0 and m1 at admission, m2 after m3's setup


@pytest.mark.parametrize("large", [10, 10 ** 6])
def test_growth_during_solves_is_charged(server_cls, large):
    make, _ = server_cls
    probs = _problems([9, 12, 15])
    grow = 5000
    S = make(grow_per_solve=grow, workers=2, large_unknowns=large)
    _register(S, probs)
    for i in range(9):
        key = f"m{i % 3}"
        S.submit(key, np.ones(probs[key].n))
    S.drain(timeout=60)
    assert _consistent(S)
    base = sum(BYTES_PER_UNKNOWN * p.n for p in probs.values())
    assert S.used == base + 9 * grow and S.max_used >= S.used
    st = S.stats()
    assert st["grown_bytes"] == 9 * grow
    S.close()


def test_rejected_matrix_fails_only_its_own_requests(server_cls):
    make, _ = server_cls
    probs = _problems([9, 12, 15])
    bad = probs["m1"]
    val = bad.val.copy()
    val[0] = -1.0  # not SPD: the library refuses it
    S = make(workers=2)
    for key, p in probs.items():
        S.register(key, p.rowptr, p.col, val if key == "m1" else p.val, p.x, p.y)
    reqs = [(k, S.submit(k, np.ones(probs[k].n))) for k in ["m0", "m1", "m2", "m1", "m0"]]
    S.drain(timeout=60)
    later = S.submit("m2", np.ones(probs["m2"].n))  # the server still serves afterwards
    S.drain(timeout=60)
    st = S.stats()
    assert _consistent(S)  # nothing stays charged for the rejected matrix
    S.close()
    for key, r in reqs + [("m2", later)]:
        assert r.done.is_set()
        if key == "m1":
            assert r.status == amg.ERR_BAD_MATRIX and r.lane == "setup" and r.x is None
        else:
            assert r.status == amg.OK and r.x is not None
    assert st["setup_failures"] >= 1 and st["setups"] == 2
    assert st["failed"] == 2 and st["completed"] == 4  # throughput counts solved requests only


def test_matrix_larger_than_the_budget_is_refused(server_cls):
    make, _ = server_cls
    big = p1_poisson(30, jitter=0.2, seed=1, rhs="normal")
    small = p1_poisson(6, jitter=0.2, seed=2, rhs="normal")
    setup_estimate = serve_module().setup_estimate

    budget = setup_estimate(small.n, len(small.col)) + 1000  # room for the small one only
    S = make(workers=1, budget_bytes=budget)
    S.register("big", big.rowptr, big.col, big.val, big.x, big.y)
    S.register("small", small.rowptr, small.col, small.val, small.x, small.y)
    r1, r2 = S.submit("big", big.b), S.submit("big", big.b)
    r3 = S.submit("small", small.b)
    S.drain(timeout=30)
    S.close()
    assert r1.status == r2.status == amg.ERR_OOM and r1.lane == "setup" and r1.x is None
    assert r3.status == amg.OK


def test_unknown_matrix_fails_its_request(server_cls):
    make, _ = server_cls
    p = p1_poisson(6, jitter=0.2, seed=2, rhs="normal")
    S = make(workers=1)
    S.register("known", p.rowptr, p.col, p.val, p.x, p.y)
    r1 = S.submit("nobody", np.ones(4))
    r2 = S.submit("known", p.b)
    S.drain(timeout=30)
    S.close()
    assert r1.status == amg.ERR_INVALID_ARG and r1.lane == "setup" and r1.x is None
    assert r2.status == amg.OK


def test_waiting_matrices_are_set_up_together(server_cls):
    """New batch-lane matrices that wait at the same time are set up by one multi-system setup
    (a large-lane matrix still on its own), each charged and resident on its own, with the
    right results."""
    make, log = server_cls
    probs = _problems([9, 12, 15, 11, 30, 10])  # m4 (784 unknowns) takes the large lane
    S = make(workers=2, large_unknowns=500)
    _register(S, probs)
    with S.cv:  # every request queued before the setup thread looks
        reqs = [(k, S.submit(k, np.ones(probs[k].n))) for k in probs]
    S.drain(timeout=60)
    st = S.stats()
    assert _consistent(S)
    S.close()
    assert log.groups == [5], log.groups
    assert st["setups"] == 6 and st["group_setups"] == 1
    for key, r in reqs:
        p = probs[key]
        assert r.status == amg.OK and r.lane == ("large" if p.n > 500 else "batch")
        np.testing.assert_allclose(r.x, _solve(p.rowptr, p.col, p.val, r.b), rtol=0, atol=1e-12)


def test_group_setup_waits_for_a_large_solve(server_cls):
    """A multi-system setup, like a single one, does not overlap a large-lane solve."""
    make, log = server_cls
    probs = _problems([30, 9, 12, 15])
    S = make(workers=1, large_unknowns=500, large_hold=0.3)
    _register(S, probs)
    S.submit("m0", np.ones(probs["m0"].n))
    _wait_running(log, "large")
    with S.cv:
        rs = [S.submit(k, np.ones(probs[k].n)) for k in ("m1", "m2", "m3")]
    S.drain(timeout=60)
    S.close()
    assert all(r.status == amg.OK for r in rs)
    assert log.groups == [3], log.groups
    assert not _overlaps(log, "large", "setup")
