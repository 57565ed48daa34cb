"""The serving loop's host tests catch plausible mistakes: each one planted in a copy of
serve.py fails at least one test of test_serve_host.py.

Each mutant is a copy of paper_1209_5421_gb300/serve.py with one mistake in the scheduling or
the memory accounting. The host tests run against it in a subprocess (through their
module-under-test hook) and must fail (pytest exit status 1). An unmodified copy must pass
through the same path.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SERVE = os.path.join(ROOT, "paper_1209_5421_gb300", "serve.py")

# name -> (text in serve.py, replacement): each text occurs exactly once
MUTANTS = {
    # admission evicts the most recently used hierarchy first
    "lru_reversed": (
        "        for key in list(self.res.keys()):",
        "        for key in reversed(list(self.res.keys())):"),
    # a request for a resident matrix does not refresh its place in the LRU order
    "no_lru_touch": (
        "                self.res.move_to_end(key)",
        "                pass"),
    # growth of a hierarchy during a solve is never charged
    "no_recharge": (
        "            nbytes = ent.h.nbytes",
        "            nbytes = ent.nbytes"),
    # no eviction when a hierarchy's real size exceeds its setup estimate
    "no_reconcile_after_setup": (
        "                self._admit(0)  # the estimate fell short: make room again (not from this one)",
        "                pass"),
    # the large lane does not wait for the running batches to drain
    "large_lane_not_exclusive": (
        "                while self.active_batches and not self.stop:  # the GPU to itself",
        "                while False:"),
    # batch workers keep launching while a large solve waits or runs
    "batches_ignore_large_lane": (
        "                    if not self.large_running and not self.large_waiting:",
        "                    if True:"),
    # setups run beside large-lane solves
    "setup_outside_grid_lock": (
        "                with self.grid_lock:\n                    h = amg.Hierarchy(",
        "                if True:\n                    h = amg.Hierarchy("),
    # multi-system setups run beside large-lane solves
    "group_setup_outside_grid_lock": (
        "            with self.grid_lock:\n                hs = amg.setup_many(",
        "            if True:\n                hs = amg.setup_many("),
    # the matrices set up with the first one are not charged before their setup
    "group_not_charged": (
        "            self.setting_up.add(k)\n            self.used += est\n",
        "            self.setting_up.add(k)\n"),
    # two requests of one matrix in one batch
    "same_system_twice_in_a_batch": (
        "            if ent is None or ent.busy or q.key in seen:",
        "            if ent is None or ent.busy:"),
    # systems routed to the wrong lane
    "lanes_swapped": (
        "            if (ent.h.n > self.large) != large:",
        "            if (ent.h.n > self.large) == large:"),
    # every request of a batch gets the first system's slice of x
    "results_misrouted": (
        "                    self._finish(q, xh[off[k]:off[k + 1]].copy(), it[k], rr[k], st[k], \"batch\")",
        "                    self._finish(q, xh[off[0]:off[1]].copy(), it[k], rr[k], st[k], \"batch\")"),
}


def _run(name, change, tmp):
    src = open(SERVE).read()
    if change is not None:
        old, new = change
        assert src.count(old) == 1, f"{name}: the mutated text must occur once in serve.py"
        src = src.replace(old, new)
    path = os.path.join(tmp, f"serve_{name}.py")
    with open(path, "w") as f:
        f.write(src)
    env = dict(os.environ, AMG_SERVE_UNDER_TEST=path)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join("tests", "test_serve_host.py"),
                        "-x", "-q", "-p", "no:cacheprovider"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    tmp = str(tmp_path_factory.mktemp("serve_mutants"))
    cases = {"unmodified": None, **MUTANTS}
    with cf.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        runs = dict(zip(cases, ex.map(lambda kv: _run(kv[0], kv[1], tmp), cases.items())))
    return runs


def test_unmodified_server_passes_through_the_same_path(results):
    rc, out = results["unmodified"]
    assert rc == 0, out


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_host_test(results, name):
    rc, out = results[name]
    assert rc == 1, f"{name}: host tests exit status {rc} (1 = a test failed)\n{out}"
