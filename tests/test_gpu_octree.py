"""GPU parity of the octree (3D) variant against the oracle, through amg_setup3.

Same bar as the quadtree: aggregates, colours, cells (t1, t2, t3), spans and level sizes
bit-exact; coarse operators row-scaled within 1e-12 with the identical stored pattern;
smoother sweeps and cycle applications within 1e-11 (FP64); solves within +-1 iteration, the
true residual at or below the tolerance, x within 1e-6 of the oracle's.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_1209_5421_gb300.meshes import p1_poisson_3d

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


def _compare(G, O):
    assert G.dim == 3 and O.dim == 3
    assert G.nlev == O.nlev and G.L == O.L
    np.testing.assert_array_equal(G.box3, np.concatenate([O.bbox, O.zbox]))
    for l in range(O.nlev):
        g, o = G.level(l), O.level(l)
        assert g["n"] == o.n and g["cellw"] == o.cellw, l
        assert g["span"] == o.span and g["m"] == o.m, l
        for k in ("t1", "t2", "t3", "color"):
            np.testing.assert_array_equal(g[k], getattr(o, k), err_msg=f"{k} level {l}")
        if l < O.nlev - 1:
            np.testing.assert_array_equal(g["agg"], o.agg)
        Ag = sp.csr_matrix((g["val"], g["col"], g["rowptr"]), shape=(g["n"], g["n"]))
        Ao = o.to_scipy()
        D = abs(Ag - Ao).tocsr()
        scale = np.asarray(abs(Ao).max(axis=1).todense()).ravel()
        assert np.all(np.asarray(D.max(axis=1).todense()).ravel() <= 1e-12 * scale), l
        np.testing.assert_array_equal(g["rowptr"], o.rowptr)
        np.testing.assert_array_equal(g["col"], o.col)


@pytest.mark.parametrize("n,opts", [(9, dict()), (17, dict(coarsest_max=8)),
                                    (33, dict()), (25, dict(aux_level=3, kcycle_n=3))])
def test_octree_setup_and_solve_parity(amg, oracle_mod, n, opts):
    p = p1_poisson_3d(n, seed=n)
    G = amg.Hierarchy.from_problem(p, **opts)
    O = oracle_mod.Hierarchy.from_problem(p, **opts)
    _compare(G, O)
    tol = 1e-8
    xg, itg, rrg, stg = G.solve(p.b, tol)
    xo, ito, _, sto = O.solve(p.b, tol)
    assert stg == amg.OK and sto == oracle_mod.OK
    assert abs(itg - ito) <= 1, (itg, ito)
    A = p.to_scipy()
    assert np.linalg.norm(p.b - A @ xg) / np.linalg.norm(p.b) <= tol
    assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)


def test_octree_smoother_and_cycle_parity(amg, oracle_mod):
    p = p1_poisson_3d(17, seed=4)
    G = amg.Hierarchy.from_problem(p, coarsest_max=8)
    O = oracle_mod.Hierarchy.from_problem(p, coarsest_max=8)
    rng = np.random.default_rng(3)
    for l in range(O.nlev):
        nl = O.level(l).n
        f = rng.standard_normal(nl)
        if l < O.nlev - 1:
            for back in (False, True):
                u0 = rng.standard_normal(nl) if back else np.zeros(nl)
                ug = G.smooth(l, f, u0, backward=back)
                uo = O.smooth(l, f, u0, backward=back)
                assert np.linalg.norm(ug - uo) <= 1e-12 * np.linalg.norm(uo), (l, back)
        zg = G.apply_cycle(l, f)
        zo = O.bhat(l, f)
        assert np.linalg.norm(zg - zo) <= 1e-11 * np.linalg.norm(zo), l


def test_octree_fp32_cycle_full(amg, oracle_mod):
    # 63^3 = 250k unknowns: the FP32 cycle with FGMRES, and with flexible CG, vs the oracle
    p = p1_poisson_3d(65, seed=1)
    O = oracle_mod.Hierarchy.from_problem(p)
    xo, ito, _, _ = O.solve(p.b, 1e-8)
    for outer in (amg.OUTER_FGMRES, amg.OUTER_FCG):
        G = amg.Hierarchy.from_problem(p, cycle_prec=amg.FP32, outer=outer)
        x, it, rr, st = G.solve(p.b, 1e-8)
        assert st == amg.OK
        A = p.to_scipy()
        assert np.linalg.norm(p.b - A @ x) / np.linalg.norm(p.b) <= 1e-8
        assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)
        assert it <= ito + 3, (it, ito)
        G.close()


def test_octree_systems_in_a_batch(amg, oracle_mod):
    # 3D hierarchies (amg_setup3) batched with a 2D one: one CTA per system, FP32 and FP64
    from paper_1209_5421_gb300.meshes import p1_poisson

    probs = [p1_poisson_3d(17, seed=1), p1_poisson(65, jitter=0.2, seed=2, rhs="normal"),
             p1_poisson_3d(33, seed=3), p1_poisson_3d(9, seed=4)]
    tol = 1e-8
    for prec in (amg.FP32, amg.FP64):
        hs = [amg.Hierarchy.from_problem(p, cycle_prec=prec) for p in probs]
        B = amg.Batch.over(hs)
        x, it, rr, st = B.solve(np.concatenate([p.b for p in probs]), tol)
        off = B.row_off
        for k, p in enumerate(probs):
            assert st[k] == amg.OK
            xk = x[off[k]:off[k + 1]]
            A = p.to_scipy()
            assert np.linalg.norm(p.b - A @ xk) / np.linalg.norm(p.b) <= tol
            xo, ito, _, _ = oracle_mod.Hierarchy.from_problem(p).solve(p.b, tol)
            assert np.linalg.norm(xk - xo) <= 1e-6 * np.linalg.norm(xo)
            assert it[k] <= ito + 3, (k, it[k], ito)
        B.close()
        for h in hs:
            h.close()


def test_octree_served(amg):
    from paper_1209_5421_gb300.serve import Server

    p = p1_poisson_3d(33, seed=5)
    S = Server(budget_bytes=1 << 30, workers=2)
    try:
        S.register("cube", p.rowptr, p.col, p.val, p.x, p.y, z=p.z)
        rng = np.random.default_rng(0)
        bs = [rng.standard_normal(p.n) for _ in range(3)]
        rs = [S.submit("cube", b) for b in bs]
        S.drain()
        A = p.to_scipy()
        for b, r in zip(bs, rs):
            assert r.status == amg.OK
            assert np.linalg.norm(b - A @ r.x) / np.linalg.norm(b) <= 1e-8
        assert S.stats()["setups"] == 1
    finally:
        S.close()


@pytest.mark.parametrize("n", [3, 5])
def test_octree_single_level_and_single_unknown(amg, oracle_mod, n):
    # 1 and 27 unknowns: one level, the exact dense solve
    p = p1_poisson_3d(n, seed=n)
    G = amg.Hierarchy.from_problem(p)
    assert G.nlev == 1 and G.dim == 3
    x, it, rr, st = G.solve(p.b, 1e-12)
    assert st == amg.OK and it == 1
    xs = np.linalg.solve(p.to_scipy().toarray(), p.b)
    assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs)
    xo, _, _, _ = oracle_mod.Hierarchy.from_problem(p).solve(p.b, 1e-12)
    assert np.linalg.norm(x - xo) <= 1e-12 * np.linalg.norm(xo)


def test_octree_invalid_inputs(amg):
    p = p1_poisson_3d(9, seed=1)
    z = p.z.copy()
    z[3] = np.nan
    with pytest.raises(amg.AmgError) as e:
        amg.Hierarchy(p.rowptr, p.col, p.val, p.x, p.y, z=z)
    assert e.value.status == amg.ERR_INVALID_ARG
    with pytest.raises(amg.AmgError) as e:  # an empty z extent
        amg.Hierarchy(p.rowptr, p.col, p.val, p.x, p.y, z=p.z, bbox=(0, 1, 0, 1, 0.5, 0.5))
    assert e.value.status == amg.ERR_INVALID_ARG
    with pytest.raises(amg.AmgError) as e:  # octree depth above 10 (2^30 cells)
        amg.Hierarchy(p.rowptr, p.col, p.val, p.x, p.y, z=p.z, aux_level=11)
    assert e.value.status == amg.ERR_UNSUPPORTED


def test_octree_full_size_cube_129(amg, oracle_mod):
    # the benchmark's 3D workload at full size (2,048,383 unknowns), FP32 cycle with FGMRES as
    # the bench times it: the hierarchy against the oracle's (sizes, cells, colours,
    # aggregates bit-exact; operators row-scaled within 1e-12), then the solve
    from paper_1209_5421_gb300.meshes import workload

    p, aux = workload("cube_129")
    G = amg.Hierarchy.from_problem(p, aux_level=aux, cycle_prec=amg.FP32, outer=amg.OUTER_FGMRES)
    O = oracle_mod.Hierarchy.from_problem(p, aux_level=aux)
    _compare(G, O)
    tol = 1e-8
    x, it, rr, st = G.solve(p.b, tol)
    xo, ito, _, sto = O.solve(p.b, tol)
    assert st == amg.OK and sto == oracle_mod.OK
    A = p.to_scipy()
    assert np.linalg.norm(p.b - A @ x) / np.linalg.norm(p.b) <= tol
    assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)
    assert it <= ito + 3, (it, ito)
    G.close()
