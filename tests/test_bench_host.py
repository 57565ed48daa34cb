"""Host logic of the benchmark and of the batched binding, on the CPU.

* bench.Clocks.summary: the SM clock median and the throttle reasons from nvidia-smi's CSV
  (the rule that rejects a run reads these);
* bench.recorded_traffic: the ncu DRAM record is reported only for the kernel sources it was
  taken on (hash of csrc/), else null;
* bench.measured_peak_hbm: the measured copy bandwidth, or the stated fallback;
* amg.Batch: the systems are concatenated into one block-diagonal CSR with row offsets, the
  layout amg_batch_setup takes; checked by reading back what reaches a stand-in library;
* bench.py --impl reference: the oracle arm's JSON line, end to end on a small workload.
"""
import ctypes as C
import json
import os
import sys

import numpy as np
import pytest
import scipy.sparse as sp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1209_5421_gb300 import amg  # noqa: E402
from paper_1209_5421_gb300.meshes import p1_poisson  # noqa: E402


def _line(sm, smax=2070, reasons=("Not Active",) * 4, active="0x0000000000000000"):
    return ", ".join(["0", str(sm), str(smax), "900.5", active, *reasons])


def test_clock_summary_median_and_reasons():
    c = bench.Clocks(0)
    c.lines = [_line(2070), _line(1980), _line(2070),
               _line(1500, reasons=("Not Active", "Not Active", "Not Active", "Active"))]
    s = c.summary()
    assert s["sm_mhz"] == 2025.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 4
    assert s["reasons"] == ["sw_power_cap"]
    c.lines.append(_line(900, reasons=("Active", "Not Active", "Active", "Not Active")))
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_clock_summary_skips_unreadable_lines():
    c = bench.Clocks(0)
    c.lines = ["", "garbage", _line("[N/A]"), "0, 2070"]
    s = c.summary()
    assert s["samples"] == 0 and s["reasons"] == ["unavailable"] and s["sm_mhz"] is None
    c.lines.append(_line(2070))
    assert c.summary()["samples"] == 1


def test_recorded_traffic_only_for_the_sources_it_was_taken_on(monkeypatch):
    with open(os.path.join(ROOT, "profiles", "cycle_traffic.json")) as f:
        rec = json.load(f)
    key, ent = next(iter(rec.items()))
    workload, prec = key.split(":")
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: ent["source_hash"])
    assert bench.recorded_traffic(workload, prec) == ent["dram_bytes_per_launch"]
    assert bench.recorded_traffic(workload, "other") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.recorded_traffic(workload, prec) is None


def test_kernel_source_hash_follows_the_sources(tmp_path, monkeypatch):
    # every file the solve kernels are compiled from changes the hash; a setup-only file not
    csrc = tmp_path / "paper_1209_5421_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        (csrc / f).write_text("x")
    (csrc / "setup.cu").write_text("x")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    (csrc / "setup.cu").write_text("y")
    assert bench.kernel_source_hash() == h0
    for f in bench.KERNEL_SOURCES:
        h1 = bench.kernel_source_hash()
        (csrc / f).write_text("y")
        assert bench.kernel_source_hash() != h1, f


def test_measured_peak_and_fallback(tmp_path, monkeypatch):
    peak, kind = bench.measured_peak_hbm()
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        assert (peak, kind) == (float(json.load(f)["hbm_gbs"]), "measured")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peak_hbm() == (6800.0, "fallback")


class _FakeLib:
    """Stands in for libamg_gb300.so: records what amg_batch_setup is given."""

    def __init__(self):
        self.seen = None

    def amg_options_default(self, o_ref):
        o = o_ref._obj
        o.aux_level, o.coarsest_max, o.kcycle_n, o.max_iters = 0, 64, 2, 200

    def amg_batch_setup(self, nprob, row_off_ptr, A_ref, x_ptr, y_ptr, o_ref, stream, b_ref):
        A = A_ref._obj
        n, nnz = A.n, A.nnz

        def arr(ptr, ctype, count):
            return np.ctypeslib.as_array((ctype * count).from_address(ptr)).copy()

        self.seen = dict(nprob=nprob, row_off=arr(row_off_ptr, C.c_int64, nprob + 1),
                         rowptr=arr(A.rowptr, C.c_int32, n + 1), col=arr(A.col, C.c_int32, nnz),
                         val=arr(A.val, C.c_double, nnz), x=arr(x_ptr, C.c_double, n),
                         y=arr(y_ptr, C.c_double, n), n=n)
        b_ref._obj.value = 1
        return amg.OK

    def amg_batch_free(self, b):
        pass


def test_batch_is_one_block_diagonal_csr(monkeypatch):
    fake = _FakeLib()
    monkeypatch.setattr(amg, "lib", lambda: fake)
    monkeypatch.setattr(amg, "_stream", lambda s: None)
    probs = [p1_poisson(n, jitter=0.2, seed=k, rhs="normal") for k, n in enumerate((9, 14, 6))]
    B = amg.Batch.from_problems(probs)
    s = fake.seen
    sizes = [p.n for p in probs]
    assert s["nprob"] == 3 and s["n"] == sum(sizes) == B.n
    np.testing.assert_array_equal(s["row_off"], np.concatenate([[0], np.cumsum(sizes)]))
    got = sp.csr_matrix((s["val"], s["col"], s["rowptr"]), shape=(s["n"], s["n"]))
    ref = sp.block_diag([p.to_scipy() for p in probs], format="csr")
    ref.sort_indices()
    np.testing.assert_array_equal(got.indptr, ref.indptr)
    np.testing.assert_array_equal(got.indices, ref.indices)
    np.testing.assert_array_equal(got.data, ref.data)
    np.testing.assert_array_equal(s["x"], np.concatenate([p.x for p in probs]))
    np.testing.assert_array_equal(s["y"], np.concatenate([p.y for p in probs]))
    B.b = None  # nothing to free in the stand-in


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the oracle, timed on the host cores) prints one JSON line
    with the contract's keys: the same metric, unit and direction as the GPU arm, its own
    cpu_baseline, and an e2e entry with no host-device traffic."""
    import subprocess

    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload",
                        "quasi_uniform_65", "--steps", "2", "--warmup", "3"], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"].startswith("solves/s")
    assert d["unit"] == "solves/s" and d["higher_is_better"] is True
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 2, 3)
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["vs_baseline"] is None
    assert d["config"]["workload"] == "quasi_uniform_65" and d["config"]["iters"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_golden_oracle_iterations_and_error():
    # the stored oracle counts (written by tests/golden/make_oracle_counts.py) are read back by
    # workload and tolerance; the error against the oracle is relative to its solution
    assert bench.golden_oracle_iters("graded_1449", 1e-8) == 126
    assert bench.golden_oracle_iters("quasi_uniform_65", 1e-8) == 10
    assert bench.golden_oracle_iters("graded_1449", 1e-6) is None
    assert bench.golden_oracle_iters("nope", 1e-8) is None
    xo = np.array([3.0, 4.0])
    assert bench.rel_err(np.array([3.0, 4.5]), xo) == pytest.approx(0.1)
