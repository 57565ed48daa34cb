"""GPU parity at the full sizes of the graded and disk workloads, against the FP64 oracle.

graded_1449: 1449^2 nodes mapped by x -> x^2, y -> y^2, coefficient jumps on 16 x 16 blocks,
2,093,809 unknowns, auxiliary depth 10 (many empty cells near (1, 1)). disk_1921: the disk of
radius 0.5 cut from the jittered 1921^2 triangulation, 2,895,245 unknowns, empty corner cells.

At these sizes the oracle's setup and one application of its preconditioner take seconds, so
the whole hierarchy is compared (aggregates, colours, cells and spans bit-exact, operators
within 1e-12 row-scaled) and one B^_0 application is compared, within the 1e-11 relative of
the small cases (observed 8e-14 on the graded mesh, 3e-14 on the disk: the two sides differ
only in the summation order of FP64 sums, and the GPU's fixed-order reductions give the same
bits on every run). The disk's oracle solve also takes seconds (iterations within +-1); the
graded mesh's takes minutes (126 iterations), so there the GPU solve is held to the oracle's
iteration count stored in tests/golden/oracle_counts.txt (within +-1) and to the true relative
residual, recomputed here in FP64 with scipy, at or below the tolerance.
"""
import numpy as np
import pytest

from paper_1209_5421_gb300.meshes import workload
from test_gpu_parity import compare_hierarchies

pytestmark = pytest.mark.gpu

TOL = 1e-8


@pytest.fixture(scope="module")
def amg():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    from paper_1209_5421_gb300 import amg as A
    from paper_1209_5421_gb300 import build

    build.build()
    return A


def _true_rel(prob, x):
    return np.linalg.norm(prob.b - prob.to_scipy() @ x) / np.linalg.norm(prob.b)


@pytest.mark.parametrize("name", ["graded_1449", "disk_1921"])
def test_full_size_hierarchy_and_cycle(amg, oracle_mod, name):
    prob, aux = workload(name)
    G = amg.Hierarchy.from_problem(prob, aux_level=aux)
    O = oracle_mod.Hierarchy.from_problem(prob, aux_level=aux)
    assert G.L == 10
    assert G.level(1)["n"] < 4 ** G.L  # empty auxiliary cells were compacted away
    compare_hierarchies(G, O)
    f = np.random.default_rng(17).standard_normal(prob.n)
    zg = G.apply_cycle(0, f)
    zo = O.bhat(0, f)
    rel = np.linalg.norm(zg - zo) / np.linalg.norm(zo)
    print(f"{name}: {G.nlev} levels, B^_0 against the oracle's: {rel:.2e}")
    assert rel <= 1e-11, rel


def test_full_size_disk_solves(amg, oracle_mod):
    prob, aux = workload("disk_1921")
    O = oracle_mod.Hierarchy.from_problem(prob, aux_level=aux)
    xo, ito, _, sto = O.solve(prob.b, TOL)
    assert sto == oracle_mod.OK
    G = amg.Hierarchy.from_problem(prob, aux_level=aux)
    x, it, rr, st = G.solve(prob.b, TOL)
    assert st == amg.OK and abs(it - ito) <= 1, (it, ito)
    assert _true_rel(prob, x) <= TOL
    assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)
    # FP32 cycle, FP64 restarted flexible GMRES: the residual bar in FP64, iterations <= + 3
    G32 = amg.Hierarchy.from_problem(prob, aux_level=aux, cycle_prec=amg.FP32,
                                     outer=amg.OUTER_FGMRES)
    x32, it32, _, st32 = G32.solve(prob.b, TOL)
    print(f"disk_1921: iterations FP64 {it}, FP32/FGMRES {it32}, oracle {ito}")
    assert st32 == amg.OK and it32 <= ito + 3, (it32, ito)
    assert _true_rel(prob, x32) <= TOL
    assert np.linalg.norm(x32 - xo) <= 1e-6 * np.linalg.norm(xo)


def test_full_size_graded_solve(amg):
    """The oracle's solve of this workload takes minutes, so its iteration count is read from
    tests/golden/oracle_counts.txt (written by a script that calls only the oracle)."""
    from test_oracle_counts import read_counts

    tol, it_oracle, _ = read_counts()["graded_1449"]
    prob, aux = workload("graded_1449")
    G = amg.Hierarchy.from_problem(prob, aux_level=aux)
    x, it, rr, st = G.solve(prob.b, tol)
    rel = _true_rel(prob, x)
    print(f"graded_1449: {it} iterations (oracle {it_oracle}), true relres {rel:.2e}")
    assert st == amg.OK, (st, it, rr)
    assert abs(it - it_oracle) <= 1, (it, it_oracle)
    assert rel <= tol
