"""Continuous-batching solve server on one GPU (resident hierarchies, HBM-budget admission).

Requests are (matrix key, right-hand side). A matrix is set up once (amg_setup) and its
hierarchy stays resident for later right-hand sides until memory is needed. Admission charges
each hierarchy's device bytes against a budget and evicts the least recently used idle
hierarchies: before its setup an estimate from the matrix's size (above the measured sizes of
2D and 3D hierarchies), after the setup and after every solve its real bytes
(amg_hierarchy_bytes; a solve can grow them, as the outer Krylov iteration allocates its
directions on demand). Where the real bytes exceed what was charged, idle hierarchies are
evicted until the total fits the budget again; the peak is reported as it was, and so are
the bytes solves added (`grown_bytes`): the peak stays within the budget plus those.

Two lanes share the GPU:
  * the batch lane: whenever systems are ready, a worker takes all of them (up to
    `max_batch`) and solves them in one persistent-kernel launch, one CTA per system, on its
    own CUDA stream (amg_batch_create over the resident hierarchies, fixed launch shape).
    Several workers run at once, so a system that becomes ready while others are on the GPU
    starts on free SMs without waiting for them: the device holds CTAs of several batches;
  * the large lane: a system above `large_unknowns` is solved by the single-system solver
    (the grid-wide cycle kernel over all SMs). It runs alone: batch workers drain first and
    wait while it runs.
Setups run on a separate thread (each on the hierarchy's own stream). New batch-lane matrices
that wait at the same time are set up together, by one multi-system setup (amg_setup_many);
each hierarchy still stands on its own (charged, evicted and freed one by one).

Every system is computed by code whose result does not depend on the other work in flight:
in the batch lane by one CTA of fixed size, in the large lane by the single-system kernel.
A request the server cannot set up ends alone, with a status (lane "setup", no x), and the
server goes on with the others: a matrix the library rejects (not SPD, invalid CSR, no device
memory) with the library's status, a matrix larger than the whole budget with ERR_OOM, a key
that was never registered with ERR_INVALID_ARG.
"""
from __future__ import annotations

import threading
import time
from collections import OrderedDict, deque
from dataclasses import dataclass, field

import numpy as np

from . import amg

# device bytes per unknown of the batched-solve workspace a hierarchy allocates on its first
# batched solve (32 FP64 directions and their images, 3 vectors, colour ranges; a system
# that needs more directions gets them on demand, and the real size replaces the estimate)
_BATCH_WS_BYTES_PER_UNKNOWN = 8 * (2 * 32 + 3)


def setup_estimate(n: int, nnz: int) -> int:
    """Device bytes charged for a hierarchy before its setup, from the fine matrix's unknowns
    and nonzeros. A stored operator entry costs 16 bytes over both precisions (int32 column,
    FP64 value, FP32 copy, 16-bit column copy); the stored entries of all levels come to about
    2.3 times the fine nonzeros in 2D and 1.3 times in 3D, plus slice padding: 64 bytes per
    fine nonzero covers them. Index maps and vectors of all levels: 200 bytes per unknown.
    Measured: about 400 bytes per unknown for the 1025 x 1025 quasi-uniform mesh, against
    650 estimated. The real size replaces the estimate after setup."""
    return int(64 * nnz + (200 + _BATCH_WS_BYTES_PER_UNKNOWN) * n)


@dataclass
class Request:
    key: object
    b: np.ndarray
    tol: float
    t_arrival: float
    lane: str = ""
    x: np.ndarray | None = None
    iters: int = -1
    relres: float = float("nan")
    status: int = -1
    t_done: float = 0.0
    done: threading.Event = field(default_factory=threading.Event)

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


class _Resident:
    def __init__(self, h: amg.Hierarchy, nbytes: int):
        self.h = h
        self.nbytes = nbytes
        self.busy = False


class Server:
    def __init__(self, budget_bytes: int = 150 << 30, cycle_prec: int = amg.FP32,
                 workers: int = 4, max_batch: int = 152, large_unknowns: int = 250_000,
                 device: int = 0, max_group: int = 64):
        import torch

        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.budget = int(budget_bytes)
        self.prec = cycle_prec
        self.max_batch = max_batch
        self.large = large_unknowns
        self.max_group = max_group  # new batch-lane matrices set up together, at most
        self.matrices: dict = {}                  # key -> (rowptr, col, val, x, y, z)
        self.res: OrderedDict = OrderedDict()      # key -> _Resident (LRU order)
        self.used = 0
        self.max_used = 0
        self.grown = 0  # bytes that solves added to resident hierarchies
        self.cv = threading.Condition()
        self.need_setup: deque = deque()           # requests whose matrix is not resident
        self.ready: deque = deque()                # requests whose hierarchy is resident
        self.setting_up: set = set()
        self.active_batches = 0
        self.large_waiting = 0
        self.large_running = False
        self.stop = False
        self.completed: list[Request] = []
        self.evictions = 0
        self.setups = 0
        self.group_setups = 0  # multi-system setups (amg_setup_many) of several matrices
        self.suspect: set = set()  # keys of a rejected group: each is set up on its own
        self.setup_failures = 0  # matrices that could not be set up (their requests failed)
        self.batches = 0
        self.errors: list[str] = []
        # setups and large-lane solves never overlap: the grid-wide kernel wants every SM
        self.grid_lock = threading.Lock()
        self.threads = [threading.Thread(target=self._setup_loop, daemon=True)]
        self.threads += [threading.Thread(target=self._batch_loop, daemon=True)
                         for _ in range(workers)]
        self.threads.append(threading.Thread(target=self._large_loop, daemon=True))
        for t in self.threads:
            t.start()

    # ---- client side ------------------------------------------------------------------
    def register(self, key, rowptr, col, val, x, y, z=None):
        """Make a matrix known to the server (host arrays); it is set up on first use.

        With `z` the nodes are points in 3D and the octree auxiliary grid aggregates them."""
        with self.cv:
            self.matrices[key] = (np.asarray(rowptr, np.int32), np.asarray(col, np.int32),
                                  np.asarray(val, np.float64), np.asarray(x, np.float64),
                                  np.asarray(y, np.float64),
                                  None if z is None else np.asarray(z, np.float64))

    def submit(self, key, b, tol: float = 1e-8) -> Request:
        r = Request(key, np.ascontiguousarray(b, np.float64), tol, time.perf_counter())
        with self.cv:
            if key in self.res:
                self.res.move_to_end(key)
                self.ready.append(r)
            else:
                self.need_setup.append(r)
            self.cv.notify_all()
        return r

    def drain(self, timeout: float = 600.0):
        """Wait until every submitted request has completed."""
        t_end = time.perf_counter() + timeout
        with self.cv:
            while self.need_setup or self.ready or self.setting_up or self.active_batches \
                    or self.large_running or self.large_waiting:
                if self.errors:
                    raise RuntimeError(self.errors[0])
                left = t_end - time.perf_counter()
                if left <= 0:
                    raise TimeoutError("server did not drain")
                self.cv.wait(min(left, 0.05))
            if self.errors:
                raise RuntimeError(self.errors[0])

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        for t in self.threads:
            t.join(timeout=60)
        for r in self.res.values():
            r.h.close()
        self.res.clear()

    def stats(self) -> dict:
        """Throughput and latency over the requests that returned a solution; requests that
        ended at setup (lane "setup") are counted apart, as `failed`."""
        solved = [r for r in self.completed if r.x is not None]
        failed = len(self.completed) - len(solved)
        lat = sorted(r.latency for r in solved)
        if not lat:
            return {"completed": 0, "failed": failed}
        t0 = min(r.t_arrival for r in solved)
        t1 = max(r.t_done for r in solved)
        return {"completed": len(lat), "failed": failed, "solves_per_s": len(lat) / (t1 - t0),
                "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                "setups": self.setups, "group_setups": self.group_setups,
                "setup_failures": self.setup_failures,
                "evictions": self.evictions, "batches": self.batches,
                "max_resident_bytes": self.max_used, "budget_bytes": self.budget,
                "grown_bytes": self.grown,
                "large_lane": sum(r.lane == "large" for r in solved)}

    # ---- internals --------------------------------------------------------------------
    def _fail(self, msg: str):
        with self.cv:
            self.errors.append(msg)
            self.cv.notify_all()

    def _finish(self, r: Request, x, it, rr, st, lane):
        r.x, r.iters, r.relres, r.status, r.lane = x, int(it), float(rr), int(st), lane
        r.t_done = time.perf_counter()
        r.done.set()
        self.completed.append(r)

    def _fail_key(self, key, status: int, first: Request | None = None):
        """End every queued request for matrix `key` (and `first`, already dequeued) with
        `status`, lane "setup", no x (caller holds cv)."""
        failed = ([first] if first is not None else []) + [q for q in self.need_setup
                                                           if q.key == key]
        for q in failed:
            if q is not first:
                self.need_setup.remove(q)
            self._finish(q, None, 0, float("nan"), status, "setup")
        self.setup_failures += 1

    def _recharge(self, ent: _Resident):
        """Charge a resident hierarchy's current bytes (a solve may have grown them) and evict
        other idle hierarchies if the total no longer fits (caller holds cv; `ent` is busy)."""
        try:
            nbytes = ent.h.nbytes
        except Exception as e:  # noqa: BLE001
            self.errors.append(f"hierarchy bytes: {e}")
            return
        if nbytes != ent.nbytes:
            self.grown += max(0, nbytes - ent.nbytes)
            self.used += nbytes - ent.nbytes
            ent.nbytes = nbytes
            self.max_used = max(self.max_used, self.used)
            self._admit(0)

    def _admit(self, need: int) -> bool:
        """Evict idle LRU hierarchies until `need` more bytes fit (caller holds cv)."""
        if need > self.budget:
            return False
        for key in list(self.res.keys()):
            if self.used + need <= self.budget:
                break
            ent = self.res[key]
            if ent.busy or any(q.key == key for q in self.ready):
                continue
            del self.res[key]
            self.used -= ent.nbytes
            self.evictions += 1
            ent.h.close()
        return self.used + need <= self.budget

    def _setup_loop(self):
        torch = self.torch
        torch.cuda.set_device(self.dev)
        while True:
            with self.cv:
                while not self.stop and not self.need_setup:
                    self.cv.wait()
                if self.stop:
                    return
                r = self.need_setup[0]
                if r.key in self.res:  # set up meanwhile for an earlier request
                    self.need_setup.popleft()
                    self.ready.append(r)
                    self.cv.notify_all()
                    continue
                m = self.matrices.get(r.key)
                if m is None:  # never registered: this request fails, the server goes on
                    self.need_setup.popleft()
                    self._finish(r, None, 0, float("nan"), amg.ERR_INVALID_ARG, "setup")
                    self.cv.notify_all()
                    continue
                n = len(m[0]) - 1
                est = setup_estimate(n, len(m[1]))  # replaced by the real bytes after setup
                while not self.stop and not self._admit(est):
                    if est > self.budget:  # can never fit: its requests fail, the rest go on
                        self._fail_key(r.key, amg.ERR_OOM)
                        self.cv.notify_all()
                        break
                    self.cv.wait(0.01)  # wait for hierarchies to become idle
                else:
                    self.need_setup.popleft()
                    self.setting_up.add(r.key)
                    self.used += est
                    self.max_used = max(self.max_used, self.used)
                if self.stop:
                    return
                if r.key not in self.setting_up:
                    continue
                group = self._companions(r, m, n)
            if group:
                done = self._setup_group(r, est, group)
                if done is None:  # an unexpected failure: the server stops
                    return
                if done:
                    continue  # else (a matrix of the group was rejected): each on its own
            h = None
            try:
                with self.grid_lock:
                    h = amg.Hierarchy(*m[:5], z=m[5], cycle_prec=self.prec,
                                      outer=amg.OUTER_FGMRES if n > self.large else amg.OUTER_FCG)
                    if n <= self.large:  # the cycle copies and batched workspace, allocated now
                        amg.Batch.over([h], threads=1024).close()
                nbytes = h.nbytes
            except (amg.AmgError, ValueError, TypeError) as e:
                # the library (or the binding) rejects this matrix: its requests end with that
                # status and the server goes on with the others
                if h is not None:
                    h.close()
                status = e.status if isinstance(e, amg.AmgError) else amg.ERR_INVALID_ARG
                with self.cv:
                    self.setting_up.discard(r.key)
                    self.used -= est
                    self._fail_key(r.key, status, first=r)
                    self.cv.notify_all()
                continue
            except Exception as e:  # noqa: BLE001
                self._fail(f"setup of {r.key!r}: {e}")
                return
            with self.cv:
                self.setting_up.discard(r.key)
                self.used += nbytes - est
                self.max_used = max(self.max_used, self.used)
                self._admit(0)  # the estimate fell short: make room again (not from this one)
                self.res[r.key] = _Resident(h, nbytes)
                self.setups += 1
                self.ready.append(r)
                # later requests for the same matrix that queued meanwhile
                for q in [q for q in self.need_setup if q.key == r.key]:
                    self.need_setup.remove(q)
                    self.ready.append(q)
                self.cv.notify_all()

    def _companions(self, r: Request, m, n: int) -> list:
        """Other new batch-lane 2D matrices waiting now, admitted at once (their estimates
        charged, marked as being set up) to be set up with r's matrix in one multi-system
        setup: [(key, estimate)], empty if none (caller holds cv)."""
        if m[5] is not None or n > self.large or self.max_group < 2 or r.key in self.suspect:
            return []
        out, seen = [], {r.key}
        for q in self.need_setup:
            if len(out) + 1 >= self.max_group:
                break
            k = q.key
            if k in seen or k in self.res or k in self.setting_up or k in self.suspect:
                continue
            mk = self.matrices.get(k)
            if mk is None or mk[5] is not None or len(mk[0]) - 1 > self.large:
                continue
            est = setup_estimate(len(mk[0]) - 1, len(mk[1]))
            if not self._admit(est):
                break
            seen.add(k)
            self.setting_up.add(k)
            self.used += est
            self.max_used = max(self.max_used, self.used)
            out.append((k, est))
        return out

    def _setup_group(self, r: Request, r_est: int, group: list) -> bool:
        """r's matrix and the group's in one amg_setup_many (each hierarchy then stands on its
        own: evicted and freed one by one). False if the library rejects the call: the
        group's charges are returned and r's setup goes on alone (each matrix of the group
        is set up later on its own, so a bad matrix fails only its own requests)."""
        keys = [r.key] + [k for k, _ in group]
        ests = dict(group)
        ests[r.key] = r_est
        try:
            with self.grid_lock:
                hs = amg.setup_many([self.matrices[k][:5] for k in keys], cycle_prec=self.prec,
                                    outer=amg.OUTER_FCG)
            sizes = [h.nbytes for h in hs]
        except (amg.AmgError, ValueError, TypeError):
            with self.cv:
                for k, est in group:
                    self.setting_up.discard(k)
                    self.used -= est
                    self.suspect.add(k)  # set up on its own from now on
                self.cv.notify_all()
            return False
        except Exception as e:  # noqa: BLE001
            self._fail(f"setup of {keys!r}: {e}")
            return None
        with self.cv:
            for k, h, nbytes in zip(keys, hs, sizes):
                self.setting_up.discard(k)
                self.used += nbytes - ests[k]
                self.res[k] = _Resident(h, nbytes)
                self.setups += 1
                if k == r.key:
                    self.ready.append(r)
                for q in [q for q in self.need_setup if q.key == k]:
                    self.need_setup.remove(q)
                    self.ready.append(q)
            self.group_setups += 1
            self.max_used = max(self.max_used, self.used)
            self._admit(0)  # estimates that fell short: make room again
            self.cv.notify_all()
        return True

    def _take_ready(self, large: bool):
        """Ready requests of one lane whose hierarchy is idle (caller holds cv)."""
        out, seen = [], set()
        for q in list(self.ready):
            ent = self.res.get(q.key)
            if ent is None or ent.busy or q.key in seen:
                continue
            if (ent.h.n > self.large) != large:
                continue
            out.append(q)
            seen.add(q.key)
            if large or len(out) >= self.max_batch:
                break
        for q in out:
            self.ready.remove(q)
            self.res[q.key].busy = True
        return out

    def _batch_loop(self):
        torch = self.torch
        torch.cuda.set_device(self.dev)
        stream = torch.cuda.Stream(self.dev)
        while True:
            with self.cv:
                while not self.stop:
                    if not self.large_running and not self.large_waiting:
                        batch = self._take_ready(large=False)
                        if batch:
                            break
                    self.cv.wait()
                if self.stop:
                    return
                self.active_batches += 1
                self.batches += 1
                hs = [self.res[q.key].h for q in batch]
            try:
                with torch.cuda.stream(stream):
                    B = amg.Batch.over(hs, threads=1024, stream=stream)
                    rhs = torch.from_numpy(np.concatenate([q.b for q in batch])).to(self.dev)
                    x, it, rr, st = B.solve(rhs, batch[0].tol if len({q.tol for q in batch}) == 1
                                            else min(q.tol for q in batch), stream=stream)
                    xh = x.cpu().numpy()
                    B.close()
                off = B.row_off
                for k, q in enumerate(batch):
                    self._finish(q, xh[off[k]:off[k + 1]].copy(), it[k], rr[k], st[k], "batch")
            except Exception as e:  # noqa: BLE001
                self._fail(f"batch solve: {e}")
                return
            finally:
                with self.cv:
                    for q in batch:
                        ent = self.res.get(q.key)
                        if ent is not None:
                            self._recharge(ent)
                    for q in batch:
                        ent = self.res.get(q.key)
                        if ent is not None:
                            ent.busy = False
                    self.active_batches -= 1
                    self.cv.notify_all()

    def _large_loop(self):
        torch = self.torch
        torch.cuda.set_device(self.dev)
        stream = torch.cuda.Stream(self.dev)
        while True:
            with self.cv:
                while not self.stop:
                    job = self._take_ready(large=True)
                    if job:
                        break
                    self.cv.wait()
                if self.stop:
                    return
                q = job[0]
                self.large_waiting += 1
                while self.active_batches and not self.stop:  # the GPU to itself
                    self.cv.wait()
                self.large_waiting -= 1
                self.large_running = True
                h = self.res[q.key].h
            try:
                with self.grid_lock, torch.cuda.stream(stream):
                    b = torch.from_numpy(q.b).to(self.dev)
                    x, it, rr, st = h.solve(b, q.tol, stream=stream)
                    xh = x.cpu().numpy()
                self._finish(q, xh, it, rr, st, "large")
            except Exception as e:  # noqa: BLE001
                self._fail(f"large solve: {e}")
                return
            finally:
                with self.cv:
                    self.large_running = False
                    ent = self.res.get(q.key)
                    if ent is not None:
                        self._recharge(ent)
                        ent.busy = False
                    self.cv.notify_all()
