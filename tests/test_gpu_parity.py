"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Bar (the method's acceptance criteria):
  * aggregates, colours, cells, spans, level sizes: bit-exact;
  * coarse operators: |dA_ij| <= 1e-12 * max_j |A_ij| (row-scaled; cancellation can leave
    exact zeros, so entrywise relative error is not meaningful);
  * smoother sweeps and cycle applications: 1e-11 relative in the 2-norm (the only
    difference is the summation order of FP64 sums);
  * solves: iteration count within +-1 of the oracle, and the true relative residual of
    the returned x, recomputed here with scipy, at or below the requested tolerance.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1209_5421_gb300.meshes import disk_poisson, five_point_grid, p1_poisson, workload

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def amg():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    from paper_1209_5421_gb300 import amg as A
    from paper_1209_5421_gb300 import build

    build.build()
    return A


def _csr(lv_rowptr, lv_col, lv_val, n):
    return sp.csr_matrix((lv_val, lv_col, lv_rowptr), shape=(n, n))


def compare_hierarchies(G, O, entry_tol=1e-12):
    assert G.nlev == O.nlev
    assert G.L == O.L
    np.testing.assert_array_equal(G.bbox, O.bbox)
    for l in range(O.nlev):
        g = G.level(l)
        o = O.level(l)
        assert g["n"] == o.n, l
        assert g["cellw"] == o.cellw, l
        assert g["span"] == o.span and g["m"] == o.m, l
        np.testing.assert_array_equal(g["t1"], o.t1)
        np.testing.assert_array_equal(g["t2"], o.t2)
        np.testing.assert_array_equal(g["color"], o.color)
        if l < O.nlev - 1:
            np.testing.assert_array_equal(g["agg"], o.agg)
        else:
            assert np.all(g["agg"] == -1)
        Ag = _csr(g["rowptr"], g["col"], g["val"], g["n"])
        Ao = o.to_scipy()
        D = (Ag - Ao).tocsr()
        rowscale = np.asarray(abs(Ao).max(axis=1).todense()).ravel()
        rowdiff = np.asarray(abs(D).max(axis=1).todense()).ravel()
        assert np.all(rowdiff <= entry_tol * rowscale), (l, (rowdiff / rowscale).max())
        # same stored pattern (every contributed (R, C) pair)
        assert g["stored"] == Ao.nnz, l
        np.testing.assert_array_equal(g["rowptr"], o.rowptr)
        np.testing.assert_array_equal(g["col"], o.col)


CASES = {
    "jitter33": (dict(n=33, jitter=0.2, seed=1, rhs="normal"), dict()),
    "quasi_uniform_65": (None, dict()),
    "graded65_kappa": (dict(n=65, jitter=0.1, graded=True, kappa_blocks=16, seed=2,
                            rhs="normal"), dict()),
    "jitter70_L5_c16": (dict(n=70, jitter=0.25, seed=3, rhs="normal"),
                        dict(aux_level=5, coarsest_max=16)),
    "kcycle3": (dict(n=41, jitter=0.2, seed=4, rhs="normal"), dict(kcycle_n=3, coarsest_max=4)),
    "kcycle1": (dict(n=41, jitter=0.2, seed=5, rhs="normal"), dict(kcycle_n=1)),
    # several smoothing sweeps (reading R10 as a parameter): 9,025 unknowns, so the finest
    # level runs grid-wide and the rest in the shared-memory tail; and a tail-only case
    "nu2": (dict(n=97, jitter=0.2, seed=6, rhs="normal"), dict(nu_pre=2, nu_post=2)),
    "nu31": (dict(n=41, jitter=0.2, seed=7, rhs="normal"), dict(nu_pre=3, nu_post=1)),
    # graded with aggregates of up to 484 unknowns: 462 above 16 (swept by warps in level
    # order), 7 above 128 (by CTAs, in shared memory in the persistent kernel)
    "graded257_kappa": (dict(n=257, jitter=0.1, graded=True, kappa_blocks=16, seed=12,
                             rhs="normal"), dict()),
}


def _problem(name):
    spec, opts = CASES[name]
    if spec is None:
        prob, aux = workload(name)
        opts = dict(opts, aux_level=aux)
    else:
        prob = p1_poisson(**spec)
    return prob, opts


@pytest.mark.parametrize("name", sorted(CASES))
def test_setup_parity(amg, oracle_mod, name):
    prob, opts = _problem(name)
    G = amg.Hierarchy.from_problem(prob, **opts)
    O = oracle_mod.Hierarchy.from_problem(prob, **opts)
    compare_hierarchies(G, O)


@pytest.mark.parametrize("name", sorted(CASES))
def test_solve_parity(amg, oracle_mod, name):
    prob, opts = _problem(name)
    G = amg.Hierarchy.from_problem(prob, **opts)
    O = oracle_mod.Hierarchy.from_problem(prob, **opts)
    tol = 1e-8
    xg, itg, rrg, stg = G.solve(prob.b, tol)
    xo, ito, rro, sto = O.solve(prob.b, tol)
    assert stg == amg.OK and sto == oracle_mod.OK
    assert abs(itg - ito) <= 1, (itg, ito)
    A = prob.to_scipy()
    true_rel = np.linalg.norm(prob.b - A @ xg) / np.linalg.norm(prob.b)
    assert true_rel <= tol and abs(true_rel - rrg) <= 1e-3 * tol
    assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)


@pytest.mark.parametrize("name", ["jitter33", "graded65_kappa", "kcycle3", "nu2", "nu31",
                                  "graded257_kappa"])
def test_smoother_and_cycle_parity(amg, oracle_mod, name):
    prob, opts = _problem(name)
    G = amg.Hierarchy.from_problem(prob, **opts)
    O = oracle_mod.Hierarchy.from_problem(prob, **opts)
    rng = np.random.default_rng(11)
    for l in range(O.nlev):
        n = O.level(l).n
        f = rng.standard_normal(n)
        if l < O.nlev - 1:
            for back in (False, True):
                u0 = rng.standard_normal(n) if back else np.zeros(n)
                ug = G.smooth(l, f, u0, backward=back)
                uo = O.smooth(l, f, u0, backward=back)
                assert np.linalg.norm(ug - uo) <= 1e-12 * np.linalg.norm(uo), (l, back)
        zg = G.apply_cycle(l, f)
        zo = O.bhat(l, f)
        assert np.linalg.norm(zg - zo) <= 1e-11 * np.linalg.norm(zo), (l, np.linalg.norm(zg - zo) / np.linalg.norm(zo))


def test_several_sweeps_fp32_cycle(amg, oracle_mod):
    # the FP32 cycle with two sweeps each way, FGMRES outer: meets the tolerance in FP64 and
    # agrees with the FP64 oracle's solution of the same preconditioned method
    prob, opts = _problem("nu2")
    G = amg.Hierarchy.from_problem(prob, cycle_prec=amg.FP32, outer=amg.OUTER_FGMRES, **opts)
    O = oracle_mod.Hierarchy.from_problem(prob, **opts)
    tol = 1e-8
    xg, itg, rrg, stg = G.solve(prob.b, tol)
    xo, ito, _, sto = O.solve(prob.b, tol)
    assert stg == amg.OK and sto == oracle_mod.OK
    A = prob.to_scipy()
    assert np.linalg.norm(prob.b - A @ xg) / np.linalg.norm(prob.b) <= tol
    assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)
    assert itg <= ito + 3, (itg, ito)
    # more sweeps than the default: fewer (or as many) outer iterations
    G1 = amg.Hierarchy.from_problem(prob, cycle_prec=amg.FP32, outer=amg.OUTER_FGMRES)
    _, it1, _, st1 = G1.solve(prob.b, tol)
    assert st1 == amg.OK and itg <= it1
    G.close()
    G1.close()


def test_graded_fp32_cycle_big_blocks(amg, oracle_mod):
    # the FP32 cycle on the graded case whose largest aggregates are swept by CTAs in shared
    # memory: meets the tolerance in FP64, agrees with the oracle's solution
    prob, opts = _problem("graded257_kappa")
    O = oracle_mod.Hierarchy.from_problem(prob, **opts)
    agg = O.level(0).agg
    assert np.bincount(agg).max() > 128
    G = amg.Hierarchy.from_problem(prob, cycle_prec=amg.FP32, outer=amg.OUTER_FGMRES, **opts)
    tol = 1e-8
    xg, itg, rrg, stg = G.solve(prob.b, tol)
    xo, ito, _, sto = O.solve(prob.b, tol)
    assert stg == amg.OK and sto == oracle_mod.OK
    A = prob.to_scipy()
    assert np.linalg.norm(prob.b - A @ xg) / np.linalg.norm(prob.b) <= tol
    assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)
    assert itg <= ito + 10, (itg, ito)
    G.close()


def test_uniform_grid_and_explicit_box(amg, oracle_mod):
    L = 5
    prob = five_point_grid(2 ** (L + 1))
    opts = dict(aux_level=L, bbox=(0.0, 1.0, 0.0, 1.0), coarsest_max=16)
    G = amg.Hierarchy.from_problem(prob, **opts)
    O = oracle_mod.Hierarchy.from_problem(prob, **opts)
    compare_hierarchies(G, O)
    x, it, rr, st = G.solve(prob.b, 1e-10)
    _, ito, _, _ = O.solve(prob.b, 1e-10)
    assert st == amg.OK and abs(it - ito) <= 1


def test_empty_cells(amg, oracle_mod):
    # graded mesh with a fine auxiliary grid leaves cells empty (aggregates are compacted)
    prob = p1_poisson(57, jitter=0.1, graded=True, seed=6, rhs="normal")
    opts = dict(aux_level=6, coarsest_max=32)
    G = amg.Hierarchy.from_problem(prob, **opts)
    O = oracle_mod.Hierarchy.from_problem(prob, **opts)
    assert G.level(1)["n"] < 4**6
    compare_hierarchies(G, O)


@pytest.mark.parametrize("n,opts", [(65, dict()), (129, dict(aux_level=7)),
                                    (257, dict(aux_level=8, cycle_prec=1))])
def test_disk_domain_parity(amg, oracle_mod, n, opts):
    # the disk cut from the square (Sec. 5 disk examples): empty auxiliary cells in the corners
    prob = disk_poisson(n, seed=n)
    gopts = dict(opts)
    oopts = {k: v for k, v in opts.items() if k != "cycle_prec"}
    G = amg.Hierarchy.from_problem(prob, **gopts)
    O = oracle_mod.Hierarchy.from_problem(prob, **oopts)
    compare_hierarchies(G, O)
    assert G.level(1)["n"] < 0.85 * 4 ** G.L
    tol = 1e-8
    xg, itg, rrg, stg = G.solve(prob.b, tol)
    xo, ito, _, _ = O.solve(prob.b, tol)
    assert stg == amg.OK and abs(itg - ito) <= (1 if "cycle_prec" not in opts else 3)
    A = prob.to_scipy()
    assert np.linalg.norm(prob.b - A @ xg) / np.linalg.norm(prob.b) <= tol
    assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)


@pytest.mark.parametrize("n,cmax", [(6, 64), (9, 49), (12, 256)])
def test_single_level_exact(amg, oracle_mod, n, cmax):
    prob = p1_poisson(n, jitter=0.2, seed=7, rhs="normal")
    G = amg.Hierarchy.from_problem(prob, coarsest_max=cmax)
    assert G.nlev == 1
    x, it, rr, st = G.solve(prob.b, 1e-12)
    assert st == amg.OK and it == 1
    xs = np.linalg.solve(prob.to_scipy().toarray(), prob.b)
    assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs)


def test_tiny_meshes_match_dense_direct(amg):
    for n in (5, 9, 13, 17):
        prob = p1_poisson(n, jitter=0.2, seed=n, rhs="normal")
        G = amg.Hierarchy.from_problem(prob, coarsest_max=4)
        x, it, rr, st = G.solve(prob.b, 1e-13)
        xs = np.linalg.solve(prob.to_scipy().toarray(), prob.b)
        assert st == amg.OK
        assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs), n


def test_deterministic_and_reusable(amg):
    prob, opts = _problem("jitter70_L5_c16")
    G = amg.Hierarchy.from_problem(prob, **opts)
    x1, it1, _, _ = G.solve(prob.b, 1e-9)
    x2, it2, _, _ = G.solve(prob.b, 1e-9)
    assert it1 == it2 and np.array_equal(x1, x2)
    G2 = amg.Hierarchy.from_problem(prob, **opts)
    x3, _, _, _ = G2.solve(prob.b, 1e-9)
    assert np.array_equal(x1, x3)
    # zero right-hand side
    x0, it0, rr0, st0 = G.solve(np.zeros(prob.n), 1e-9)
    assert st0 == amg.OK and it0 == 0 and np.all(x0 == 0)


def test_device_and_host_buffers_agree(amg):
    import torch

    prob, opts = _problem("jitter33")
    dev = "cuda"
    t = lambda a: torch.as_tensor(a).to(dev)  # noqa: E731
    Gd = amg.Hierarchy(t(prob.rowptr), t(prob.col), t(prob.val), t(prob.x), t(prob.y), **opts)
    Gh = amg.Hierarchy.from_problem(prob, **opts)
    xd, itd, _, _ = Gd.solve(t(prob.b), 1e-9)
    xh, ith, _, _ = Gh.solve(prob.b, 1e-9)
    assert itd == ith and np.array_equal(xd.cpu().numpy(), xh)


def test_invalid_inputs(amg):
    prob = p1_poisson(9, jitter=0.2)
    col = prob.col.copy()
    col[[1, 2]] = col[[2, 1]]
    with pytest.raises(amg.AmgError) as e:
        amg.Hierarchy(prob.rowptr, col, prob.val, prob.x, prob.y)
    assert e.value.status == amg.ERR_BAD_MATRIX
    val = prob.val.copy()
    val[0] = -1.0
    with pytest.raises(amg.AmgError) as e:
        amg.Hierarchy(prob.rowptr, prob.col, val, prob.x, prob.y)
    assert e.value.status == amg.ERR_BAD_MATRIX
    x = prob.x.copy()
    x[4] = np.inf
    with pytest.raises(amg.AmgError) as e:
        amg.Hierarchy(prob.rowptr, prob.col, prob.val, x, prob.y)
    assert e.value.status == amg.ERR_INVALID_ARG
    with pytest.raises(amg.AmgError) as e:
        amg.Hierarchy.from_problem(prob, coarsest_max=100000)
    assert e.value.status == amg.ERR_UNSUPPORTED
    G = amg.Hierarchy.from_problem(prob, max_iters=1, coarsest_max=4)
    x, it, rr, st = G.solve(prob.b, 1e-14)
    assert st == amg.ERR_NOT_CONVERGED and it == 1 and rr > 1e-14


def _read_golden(name):
    d = {}
    for line in open(os.path.join(HERE, "golden", name)):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        d[k] = [float(t) for t in v]
    return d


def test_ell_worked_example(amg):
    g = _read_golden("ell_example.txt")
    rows, width = int(g["rows"][0]), int(g["width"][0])
    Aj, Ax = amg.csr_to_ell(np.array(g["rowptr"], np.int32), np.array(g["col"], np.int32),
                            np.array(g["val"]), width, diag_first=False)
    np.testing.assert_array_equal(Aj, np.array(g["Aj"], np.int32))
    np.testing.assert_array_equal(Ax, np.array(g["Ax"]))
    # diagonal-first storage (Sec. 4.1, last paragraph): row 1 becomes [1, 0, 2]
    Aj, Ax = amg.csr_to_ell(np.array(g["rowptr"], np.int32), np.array(g["col"], np.int32),
                            np.array(g["val"]), width, diag_first=True)
    np.testing.assert_array_equal(Aj.reshape(width, rows).T, [[0, 1, -1], [1, 0, 2], [2, 3, -1]])
    np.testing.assert_array_equal(Ax.reshape(width, rows).T, [[4, -2, 0], [2, -1, -1], [-3, 4, 0]])
    with pytest.raises(amg.AmgError):
        amg.csr_to_ell(np.array(g["rowptr"], np.int32), np.array(g["col"], np.int32),
                       np.array(g["val"]), 2)


def test_full_size_quasi_uniform_parity(amg, oracle_mod):
    """The 1025 x 1025 quasi-uniform workload at full size, in the launch configuration the
    benchmark times (FP64 cycle, flexible CG outer): bit-exact aggregates, colours and spans on
    every level, coarse operators within 1e-12 (row-scaled), iteration count within +-1."""
    prob, aux = workload("quasi_uniform_1025")
    G = amg.Hierarchy.from_problem(prob, aux_level=aux)
    O = oracle_mod.Hierarchy.from_problem(prob, aux_level=aux)
    compare_hierarchies(G, O)
    x, it, rr, st = G.solve(prob.b, 1e-8)
    xo, ito, rro, sto = O.solve(prob.b, 1e-8)
    assert st == amg.OK and abs(it - ito) <= 1, (it, ito)
    A = prob.to_scipy()
    assert np.linalg.norm(prob.b - A @ x) / np.linalg.norm(prob.b) <= 1e-8
