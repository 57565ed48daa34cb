"""GPU: batched systems (amg_batch_setup / amg_batch_solve) against the oracle.

Every system of a batch is solved by one CTA of one persistent kernel with the same
hierarchy amg_setup builds. Each system's solution must meet the tolerance in FP64 (true
residual recomputed here), agree with the oracle's solution as closely as two converged
solves of the same system can (1e-6 relative, the bound the FP32-cycle tests use), take about
the oracle's number of outer iterations, and be the same when the system is solved alone.
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
    return A


# uneven sizes, a graded mesh with coefficient jumps, and a system small enough to have one
# level (its "cycle" is the exact dense solve)
SPECS = [
    dict(n=65, jitter=0.2, seed=0, rhs="normal"),
    dict(n=17, jitter=0.2, seed=1, rhs="normal"),
    dict(n=97, jitter=0.1, graded=True, kappa_blocks=16, seed=2, rhs="normal"),
    dict(n=45, jitter=0.2, seed=3, rhs="normal"),
    dict(n=6, jitter=0.1, seed=4, rhs="normal"),
    dict(n=129, jitter=0.2, seed=5, rhs="normal"),
]


def _check_system(amg, oracle_mod, prob, x, it, rr, st, tol, slack):
    assert st == amg.OK, st
    A = prob.to_scipy()
    true_rel = np.linalg.norm(prob.b - A @ x) / np.linalg.norm(prob.b)
    assert true_rel <= tol, true_rel
    assert abs(rr - true_rel) <= 1e-3 * tol + 1e-14, (rr, true_rel)
    O = oracle_mod.Hierarchy.from_problem(prob)
    xo, ito, _, _ = O.solve(prob.b, tol)
    err = np.linalg.norm(x - xo) / np.linalg.norm(xo)
    assert err <= 1e-6, err
    if slack is None:
        # the plain FP64 method: the same flexible CG as the oracle, so within one iteration
        assert abs(int(it) - int(ito)) <= 1, (it, ito)
    else:
        assert it <= ito + slack, (it, ito)
    return err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_matches_oracle(amg, oracle_mod, prec):
    probs = [p1_poisson(**s) for s in SPECS]
    cp = amg.FP32 if prec == "fp32" else amg.FP64
    B = amg.Batch.from_problems(probs, cycle_prec=cp)
    rhs = np.concatenate([p.b for p in probs])
    tol = 1e-8
    x, it, rr, st = B.solve(rhs, tol)
    info = B.info()
    assert info["nprob"] == len(probs) and info["threads"] in (256, 512, 1024)
    assert info["ctas"] >= 1 and info["bytes"] > 0
    off = B.row_off
    for k, p in enumerate(probs):
        # FP32 cycles: the rounding of the cycle may cost a few iterations more than the
        # FP64 oracle's; the FP64 cycle is held to the oracle's count within one
        slack = None if prec == "fp64" else (10 if SPECS[k].get("graded") else 3)
        _check_system(amg, oracle_mod, p, x[off[k]:off[k + 1]], it[k], rr[k], st[k], tol, slack)
    # a second solve replays the captured launch: same bits
    x2, it2, _, _ = B.solve(rhs, tol)
    assert np.array_equal(x2, x) and np.array_equal(it2, it)
    B.close()


def test_batch_several_sweeps_matches_oracle(amg, oracle_mod):
    # two sweeps each way on every level (reading R10 as a parameter), the plain FP64 method:
    # within one iteration of the oracle's count with the same sweeps
    probs = [p1_poisson(**s) for s in SPECS[:4]]
    B = amg.Batch.from_problems(probs, cycle_prec=amg.FP64, nu_pre=2, nu_post=2)
    rhs = np.concatenate([p.b for p in probs])
    tol = 1e-8
    x, it, rr, st = B.solve(rhs, tol)
    off = B.row_off
    for k, p in enumerate(probs):
        assert st[k] == amg.OK
        A = p.to_scipy()
        xk = x[off[k]:off[k + 1]]
        assert np.linalg.norm(p.b - A @ xk) / np.linalg.norm(p.b) <= tol
        O = oracle_mod.Hierarchy.from_problem(p, nu_pre=2, nu_post=2)
        xo, ito, _, _ = O.solve(p.b, tol)
        assert abs(int(it[k]) - int(ito)) <= 1, (k, it[k], ito)
        assert np.linalg.norm(xk - xo) <= 1e-6 * np.linalg.norm(xo)
    B.close()


def test_system_alone_and_in_the_batch(amg):
    probs = [p1_poisson(**s) for s in SPECS]
    tol = 1e-8
    B = amg.Batch.from_problems(probs, cycle_prec=amg.FP32)
    xb, itb, _, _ = B.solve(np.concatenate([p.b for p in probs]), tol)
    off = B.row_off
    for k in (0, 2):
        alone = amg.Batch.from_problems([probs[k]], cycle_prec=amg.FP32)
        xa, ita, _, sta = alone.solve(probs[k].b, tol)
        assert sta[0] == amg.OK
        xk = xb[off[k]:off[k + 1]]
        assert np.linalg.norm(xa - xk) / np.linalg.norm(xk) <= 1e-6
        assert abs(int(ita[0]) - int(itb[k])) <= 1
        # and against the single-system solver on the same system
        H = amg.Hierarchy.from_problem(probs[k], cycle_prec=amg.FP32)
        xs, its, _, sts = H.solve(probs[k].b, tol)
        assert sts == amg.OK
        assert np.linalg.norm(xs - xk) / np.linalg.norm(xk) <= 1e-6
        assert abs(its - int(itb[k])) <= 1
        alone.close()
        H.close()
    B.close()


def test_batch_device_buffers_and_zero_rhs(amg):
    import torch

    probs = [p1_poisson(**s) for s in SPECS[:4]]
    B = amg.Batch.from_problems(probs, cycle_prec=amg.FP32, device="cuda")
    rhs = np.concatenate([p.b for p in probs])
    off = B.row_off
    rhs[off[1]:off[2]] = 0.0  # system 1 has b = 0: x = 0 after no iteration
    xd, it, rr, st = B.solve(torch.as_tensor(rhs).cuda(), 1e-8)
    x = xd.cpu().numpy()
    assert (st == amg.OK).all()
    assert it[1] == 0 and rr[1] == 0.0 and not x[off[1]:off[2]].any()
    xh, ith, _, _ = B.solve(rhs, 1e-8)  # host buffers: the same numbers
    assert np.array_equal(xh, x) and np.array_equal(ith, it)
    B.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_teams_match_oracle_and_one_cta(amg, oracle_mod, prec):
    # an autotuned batch sizes teams of CTAs for its largest systems: with these few systems
    # on a full grid every system above 4 rows per thread gets a team
    probs = [p1_poisson(**s) for s in SPECS] + [p1_poisson(n=257, jitter=0.2, seed=9, rhs="normal")]
    cp = amg.FP32 if prec == "fp32" else amg.FP64
    B = amg.Batch.from_problems(probs, cycle_prec=cp)
    rhs = np.concatenate([p.b for p in probs])
    tol = 1e-8
    x, it, rr, st = B.solve(rhs, tol)
    teams = B.teams()
    assert teams.max() > 1 and teams.min() >= 1 and teams.max() <= 8
    assert teams[-1] == teams.max()  # the largest system has the largest team
    off = B.row_off
    for k, p in enumerate(probs):
        slack = None if prec == "fp64" else (10 if k < len(SPECS) and SPECS[k].get("graded") else 3)
        _check_system(amg, oracle_mod, p, x[off[k]:off[k + 1]], it[k], rr[k], st[k], tol, slack)
    # the same bits again (team sums in rank order)
    x2, it2, _, _ = B.solve(rhs, tol)
    assert np.array_equal(x2, x) and np.array_equal(it2, it)
    # one CTA per system: the same solutions up to rounding, about the same iterations
    B.set_teams(1)
    x1, it1, _, st1 = B.solve(rhs, tol)
    assert (st1 == amg.OK).all() and (B.teams() == 1).all()
    for k in range(len(probs)):
        xs, xt = x1[off[k]:off[k + 1]], x[off[k]:off[k + 1]]
        assert np.linalg.norm(xs - xt) <= 1e-6 * np.linalg.norm(xs)
        assert abs(int(it1[k]) - int(it[k])) <= 1
    # a cap on the team size
    B.set_teams(2)
    x3, _, _, st3 = B.solve(rhs, tol)
    assert (st3 == amg.OK).all() and B.teams().max() == 2
    B.close()


def test_fixed_shape_has_no_teams(amg):
    probs = [p1_poisson(**s) for s in SPECS[:3]]
    hs = [amg.Hierarchy.from_problem(p, cycle_prec=amg.FP32) for p in probs]
    B = amg.Batch.over(hs, threads=1024)
    B.solve(np.concatenate([p.b for p in probs]), 1e-8)
    assert (B.teams() == 1).all()
    B.set_teams(4)  # allowed explicitly: the batch's systems then form teams
    _, _, _, st = B.solve(np.concatenate([p.b for p in probs]), 1e-8)
    assert (st == amg.OK).all() and B.teams().max() > 1
    B.close()
    for h in hs:
        h.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_with_a_single_unknown_system(amg, prec):
    # a one-unknown system (one level, exact solve) beside a large one that forms a team
    probs = [p1_poisson(n=3, jitter=0.2, seed=1, rhs="normal"),
             p1_poisson(n=129, jitter=0.2, seed=2, rhs="normal")]
    cp = amg.FP32 if prec == "fp32" else amg.FP64
    B = amg.Batch.from_problems(probs, cycle_prec=cp)
    x, it, rr, st = B.solve(np.concatenate([p.b for p in probs]), 1e-8)
    assert (st == amg.OK).all()
    off = B.row_off
    assert x[0] == pytest.approx(probs[0].b[0] / probs[0].val[0], rel=1e-12)
    A = probs[1].to_scipy()
    x1 = x[off[1]:off[2]]
    assert np.linalg.norm(probs[1].b - A @ x1) / np.linalg.norm(probs[1].b) <= 1e-8
    assert B.teams()[1] > 1 and B.teams()[0] == 1
    B.close()


def test_full_batch_workload(amg, oracle_mod):
    # the benchmark's batched configuration at full size: 256 systems (13M unknowns), FP32
    # cycle, autotuned launch shape with teams. Every system meets the FP64 true residual;
    # every 32nd system is compared with the oracle's solution one by one.
    from paper_1209_5421_gb300.meshes import batch_workload

    probs = batch_workload()
    B = amg.Batch.from_problems(probs, cycle_prec=amg.FP32)
    tol = 1e-8
    x, it, rr, st = B.solve(np.concatenate([p.b for p in probs]), tol)
    assert (st == amg.OK).all()
    assert B.teams().max() > 1
    off = B.row_off
    for k, p in enumerate(probs):
        xk = x[off[k]:off[k + 1]]
        A = p.to_scipy()
        assert np.linalg.norm(p.b - A @ xk) / np.linalg.norm(p.b) <= tol, k
    for k in range(0, len(probs), 32):
        _check_system(amg, oracle_mod, probs[k], x[off[k]:off[k + 1]], it[k], rr[k], st[k], tol, 3)
    B.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_setup_matches_single_setups(amg, prec):
    # amg_batch_setup builds every system of more than coarsest_max unknowns with one set of
    # multi-system kernels (the one-level systems with the single-system setup): each
    # hierarchy must be the one the single-system setup builds, bit for bit (levels,
    # operators, aggregates, colours), and so must everything its solves read (reciprocal
    # diagonals, FP32 copies, big-block schedules, level tables): a fixed-shape batch over the
    # batched setup's hierarchies and one over single setups give the same bits, and so do
    # single-system solves of the same system
    probs = [p1_poisson(**s) for s in SPECS] + [p1_poisson(n=129, jitter=0.1, graded=True,
                                                           kappa_blocks=16, seed=11)]
    cp = amg.FP32 if prec == "fp32" else amg.FP64
    B = amg.Batch.from_problems(probs, cycle_prec=cp)
    singles = [amg.Hierarchy.from_problem(p, cycle_prec=cp) for p in probs]
    for k, p in enumerate(probs):
        Gb, Gs = B.system(k), singles[k]
        assert Gb.nlev == Gs.nlev, k
        assert np.array_equal(Gb.bbox, Gs.bbox) and Gb.L == Gs.L, k
        for l in range(Gs.nlev):
            assert Gb.level_info(l) == Gs.level_info(l), (k, l)
            lb, ls = Gb.level(l), Gs.level(l)
            for key in ls:
                np.testing.assert_array_equal(lb[key], ls[key], err_msg=f"system {k} level {l} {key}")
    rhs = [np.random.default_rng(k).standard_normal(p.n) for k, p in enumerate(probs)]
    views = [B.system(k) for k in range(len(probs))]
    Bb = amg.Batch.over(views, threads=1024)
    Bs = amg.Batch.over(singles, threads=1024)
    xb, itb, rrb, stb = Bb.solve(np.concatenate(rhs), 1e-8)
    xs, its, rrs, sts = Bs.solve(np.concatenate(rhs), 1e-8)
    assert (stb == amg.OK).all() and (sts == amg.OK).all()
    np.testing.assert_array_equal(xb, xs)
    np.testing.assert_array_equal(itb, its)
    Bb.close()
    Bs.close()
    for k in (1, 5, 6):  # the single-system solver on a batch's system (its engine built then)
        x1, it1, _, st1 = views[k].solve(rhs[k], 1e-8)
        x2, it2, _, st2 = singles[k].solve(rhs[k], 1e-8)
        assert st1 == amg.OK and st2 == amg.OK and it1 == it2, k
        np.testing.assert_array_equal(x1, x2)
    for G in singles:
        G.close()
    B.close()


@pytest.mark.parametrize("opts", [dict(coarsest_max=16, kcycle_n=3),
                                  dict(aux_level=5, bbox=(0.0, 1.0, 0.0, 1.0), coarsest_max=8),
                                  dict(nu_pre=2, nu_post=3, coarsest_max=256)])
def test_batched_setup_options_match_single_setups(amg, opts):
    # the options reach every system of the batched setup as they reach amg_setup: a fixed
    # depth and box (levels of every system from the same auxiliary grid), a small or large
    # coarsest level (with coarsest_max 256 a 225-unknown system is its own coarsest level, and
    # the others factor coarsest levels of more than 102 rows in global memory)
    probs = [p1_poisson(n=n, jitter=0.2, seed=20 + n, rhs="normal") for n in (17, 33, 65, 40)]
    B = amg.Batch.from_problems(probs, **opts)
    for k, p in enumerate(probs):
        Gb, Gs = B.system(k), amg.Hierarchy.from_problem(p, **opts)
        assert Gb.nlev == Gs.nlev and Gb.L == Gs.L, k
        assert np.array_equal(Gb.bbox, Gs.bbox), k
        for l in range(Gs.nlev):
            assert Gb.level_info(l) == Gs.level_info(l), (k, l)
            lb, ls = Gb.level(l), Gs.level(l)
            for key in ls:
                np.testing.assert_array_equal(lb[key], ls[key], err_msg=f"system {k} level {l} {key}")
        Gs.close()
    x, it, rr, st = B.solve(np.concatenate([p.b for p in probs]), 1e-8)
    assert (st == amg.OK).all() and (rr <= 1e-8).all()
    B.close()


def test_batched_setup_rejects_a_bad_system(amg):
    # one invalid system fails the whole call with amg_setup's status, and nothing leaks
    import torch

    probs = [p1_poisson(n=n, jitter=0.2, seed=n, rhs="normal") for n in (33, 17, 45)]
    B = amg.Batch.from_problems(probs)
    B.close()
    torch.cuda.synchronize()
    base = amg.pool_bytes_in_use(torch.cuda.current_device())
    sysl = [(p.rowptr, p.col, p.val, p.x, p.y) for p in probs]
    bad_val = probs[1].val.copy()
    bad_val[0] = -1.0  # a non-positive diagonal
    bad_col = probs[2].col.copy()
    bad_col[[1, 2]] = bad_col[[2, 1]]  # unsorted columns
    bad_x = probs[1].x.copy()
    bad_x[3] = np.nan
    cases = [(1, 2, bad_val, amg.ERR_BAD_MATRIX), (2, 1, bad_col, amg.ERR_BAD_MATRIX),
             (1, 3, bad_x, amg.ERR_INVALID_ARG)]
    for k, field, arr, status in cases:
        probl = list(sysl)
        t = list(probl[k])
        t[field] = arr
        probl[k] = tuple(t)
        with pytest.raises(amg.AmgError) as e:
            amg.Batch(probl)
        assert e.value.status == status, (k, field)
        torch.cuda.synchronize()
        assert amg.pool_bytes_in_use(torch.cuda.current_device()) == base
    B = amg.Batch(sysl)  # the library goes on
    x, it, rr, st = B.solve(np.concatenate([p.b for p in probs]), 1e-8)
    assert (st == amg.OK).all()
    B.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_graded_systems_big_aggregates(amg, oracle_mod, prec):
    # graded meshes: aggregates of up to 484 unknowns on the finest level (462 above 16
    # unknowns, a warp's in level order; 8 above 128, a CTA's). Alone on a CTA, in a team of
    # CTAs and in teams of at most 2: the FP64 cycle within one iteration of the oracle
    probs = [p1_poisson(n=257, jitter=0.1, graded=True, kappa_blocks=16, seed=12, rhs="normal"),
             p1_poisson(n=97, jitter=0.1, graded=True, kappa_blocks=16, seed=2, rhs="normal"),
             p1_poisson(n=193, jitter=0.1, graded=True, kappa_blocks=16, seed=13, rhs="normal")]
    for p in probs:
        agg = oracle_mod.Hierarchy.from_problem(p).level(0).agg
        assert np.bincount(agg).max() > 128 or p.n < 10000
    cp = amg.FP32 if prec == "fp32" else amg.FP64
    B = amg.Batch.from_problems(probs, cycle_prec=cp)
    rhs = np.concatenate([p.b for p in probs])
    tol = 1e-8
    off = B.row_off
    for cap in (None, 1, 2):
        if cap is not None:
            B.set_teams(cap)
        x, it, rr, st = B.solve(rhs, tol)
        if cap is None:
            assert B.teams().max() > 1
        for k, p in enumerate(probs):
            slack = None if prec == "fp64" else 10
            _check_system(amg, oracle_mod, p, x[off[k]:off[k + 1]], it[k], rr[k], st[k], tol,
                          slack)
    B.close()


def test_directions_grow_to_max_iters(amg, oracle_mod):
    # a system needing more outer directions than a batch allocates at first (32) gets more in
    # a further launch and keeps all of them: the same iterates as the oracle's unbounded
    # flexible CG. With max_iters = 40 it stops there, not converged, with a valid x.
    p = p1_poisson(n=193, jitter=0.1, graded=True, kappa_blocks=16, seed=13, rhs="normal")
    q = p1_poisson(n=33, jitter=0.2, seed=3, rhs="normal")
    B = amg.Batch.from_problems([p, q], cycle_prec=amg.FP64, max_iters=40)
    x, it, rr, st = B.solve(np.concatenate([p.b, q.b]), 1e-8)
    assert st[0] == amg.ERR_NOT_CONVERGED and it[0] == 40, (st, it)
    assert st[1] == amg.OK
    xp = x[:p.n]
    true_rel = np.linalg.norm(p.b - p.to_scipy() @ xp) / np.linalg.norm(p.b)
    assert abs(rr[0] - true_rel) <= 1e-6 * true_rel, (rr[0], true_rel)
    assert 1e-8 < true_rel < 1.0
    # the oracle's iterate after 40 steps: the same residual up to rounding
    O = oracle_mod.Hierarchy.from_problem(p, max_iters=40)
    xo, ito, rro, _ = O.solve(p.b, 1e-8)
    assert ito == 40
    assert abs(true_rel - rro) <= 1e-3 * rro, (true_rel, rro)
    # a second solve starts with the grown workspace: the same result
    x2, it2, _, st2 = B.solve(np.concatenate([p.b, q.b]), 1e-8)
    assert np.array_equal(x2, x) and np.array_equal(it2, it) and np.array_equal(st2, st)
    B.close()


def test_moved_bytes_of_a_batch(amg):
    # amg_batch_moved_bytes: 0 before a solve; with a fixed shape each system's solve does not
    # depend on the others, so the batch's bytes are the sum of its systems' alone; and a
    # system's bytes exceed its outer steps times one cycle application's stored matrix entries
    probs = [p1_poisson(n=n, jitter=0.2, seed=30 + n, rhs="normal") for n in (33, 65)]
    hs = [amg.Hierarchy.from_problem(p, cycle_prec=amg.FP32) for p in probs]
    both = amg.Batch.over(hs, threads=1024)
    assert both.moved_bytes() == 0.0
    _, it2, _, st2 = both.solve(np.concatenate([p.b for p in probs]), 1e-8)
    b2 = both.moved_bytes()
    both.close()
    alone = []
    for k, h in enumerate(hs):
        B = amg.Batch.over([h], threads=1024)
        _, it1, _, st1 = B.solve(probs[k].b, 1e-8)
        assert st1[0] == amg.OK and it1[0] == it2[k]
        alone.append(B.moved_bytes())
        nnz = sum(h.level_info(l)["stored"] for l in range(h.nlev))
        assert alone[-1] > it1[0] * nnz * 8  # every level's entries (4-byte index, FP32 value)
        B.close()
    assert (st2 == amg.OK).all()
    assert b2 == pytest.approx(alone[0] + alone[1], rel=1e-12)
    for h in hs:
        h.close()


@pytest.mark.parametrize("outer", ["fcg", "fgmres"])
def test_setup_many_gives_independent_single_hierarchies(amg, outer):
    # amg_setup_many: the batched setup's hierarchies returned one by one, each the one
    # amg_setup builds (bit for bit, solves included), each freed on its own
    import torch

    kw = dict(cycle_prec=amg.FP32, outer=amg.OUTER_FGMRES) if outer == "fgmres" else {}
    probs = [p1_poisson(**s) for s in SPECS] + [p1_poisson(n=129, jitter=0.1, graded=True,
                                                           kappa_blocks=16, seed=11, rhs="normal")]
    torch.cuda.synchronize()
    base = amg.pool_bytes_in_use(torch.cuda.current_device())
    many = amg.setup_many([(p.rowptr, p.col, p.val, p.x, p.y) for p in probs], **kw)
    singles = [amg.Hierarchy.from_problem(p, **kw) for p in probs]
    for k, (Gm, Gs) in enumerate(zip(many, singles)):
        assert Gm.nlev == Gs.nlev and Gm.L == Gs.L, k
        for l in range(Gs.nlev):
            assert Gm.level_info(l) == Gs.level_info(l), (k, l)
            lm, ls = Gm.level(l), Gs.level(l)
            for key in ls:
                np.testing.assert_array_equal(lm[key], ls[key], err_msg=f"system {k} level {l} {key}")
    many[0].close()  # one freed: the others are untouched
    for k in range(1, len(probs)):
        x1, it1, _, st1 = many[k].solve(probs[k].b, 1e-8)
        x2, it2, _, st2 = singles[k].solve(probs[k].b, 1e-8)
        assert st1 == amg.OK and st2 == amg.OK and it1 == it2, k
        np.testing.assert_array_equal(x1, x2)
    if outer == "fcg":  # ready for batched solves: the same bits as over single setups
        rhs = np.concatenate([p.b for p in probs[1:]])
        Bm = amg.Batch.over(many[1:], threads=1024)
        Bs = amg.Batch.over(singles[1:], threads=1024)
        xm, itm, _, stm = Bm.solve(rhs, 1e-8)
        xs, its, _, sts = Bs.solve(rhs, 1e-8)
        assert (stm == amg.OK).all()
        np.testing.assert_array_equal(xm, xs)
        np.testing.assert_array_equal(itm, its)
        Bm.close()
        Bs.close()
    for G in many[1:] + singles:
        G.close()
    torch.cuda.synchronize()
    assert amg.pool_bytes_in_use(torch.cuda.current_device()) == base
