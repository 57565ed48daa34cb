"""The stored oracle iteration counts (tests/golden/oracle_counts.txt) are the oracle's.

The file is written by tests/golden/make_oracle_counts.py, which calls only oracle/. Its
cheap entries are recomputed here; the expensive ones (minutes of oracle time) are what the
full-size GPU tests compare against.
"""
import os

import numpy as np
import pytest

from paper_1209_5421_gb300.meshes import workload

HERE = os.path.dirname(os.path.abspath(__file__))
CHEAP = {"quasi_uniform_65"}


def read_counts():
    out = {}
    with open(os.path.join(HERE, "golden", "oracle_counts.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, tol, it, rel = line.split()
            out[name] = (float(tol), int(it), float(rel))
    return out


def test_file_lists_the_full_size_workloads():
    c = read_counts()
    assert "graded_1449" in c and CHEAP <= set(c)
    for tol, it, rel in c.values():
        assert it > 0 and 0 < rel <= tol


@pytest.mark.parametrize("name", sorted(CHEAP))
def test_cheap_entries_recomputed(oracle_mod, name):
    tol, it, rel = read_counts()[name]
    prob, aux = workload(name)
    h = oracle_mod.Hierarchy.from_problem(prob, aux_level=aux)
    x, it2, rr, st = h.solve(prob.b, tol)
    assert st == oracle_mod.OK and it2 == it
    true = np.linalg.norm(prob.b - prob.to_scipy() @ x) / np.linalg.norm(prob.b)
    assert abs(true - rel) <= 1e-6 * rel
