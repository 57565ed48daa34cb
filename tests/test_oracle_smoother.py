"""Pins of the oracle's quadtree colouring and colored Gauss-Seidel smoother (Sec. 4.5).

Spans, colours and the sweep order are recomputed here in numpy from the cells and the
pattern; the sweeps are checked against dense triangular solves of the permuted matrix:
a forward Gauss-Seidel sweep from zero is (D + L_pi)^{-1} f, and a backward sweep from u2 is
u2 + (D + U_pi)^{-1} (f - A u2).
"""
import numpy as np
import pytest
import scipy.linalg as sla

from paper_1209_5421_gb300.meshes import five_point_grid, p1_poisson

CASES = [
    dict(n=17, jitter=0.2, seed=0),
    dict(n=23, jitter=0.1, graded=True, kappa_blocks=16, seed=3),
    dict(n=21, jitter=0.25, seed=9),
]


def _span(lv):
    rows = np.repeat(np.arange(lv.n), np.diff(lv.rowptr))
    return int(max(np.abs(lv.t1[rows] - lv.t1[lv.col]).max(),
                   np.abs(lv.t2[rows] - lv.t2[lv.col]).max()))


@pytest.mark.parametrize("case", CASES)
def test_span_colours_and_order(oracle_mod, case):
    prob = p1_poisson(**case)
    h = oracle_mod.Hierarchy.from_problem(prob, coarsest_max=4)
    for l in range(h.nlev - 1):
        lv = h.level(l)
        s = _span(lv)
        assert lv.span == s
        m = max(2, s + 1)
        assert lv.m == m
        np.testing.assert_array_equal(lv.color, lv.t1 % m + m * (lv.t2 % m))
        block = lv.agg if l == 0 else np.arange(lv.n)
        # colour ascending, then block (aggregate / cell) ascending, then row ascending
        np.testing.assert_array_equal(lv.perm, np.lexsort((np.arange(lv.n), block, lv.color)))
        # blocks of one colour are never coupled: every off-block entry joins two colours
        rows = np.repeat(np.arange(lv.n), np.diff(lv.rowptr))
        other = block[rows] != block[lv.col]
        assert np.all(lv.color[rows][other] != lv.color[lv.col][other])
        # a fine block is the set of unknowns in one level-L cell
        if l == 0:
            cell = lv.t1 + lv.cellw * lv.t2
            assert np.all((cell[rows] == cell[lv.col]) == ~other)


@pytest.mark.parametrize("vertical", [True, False])
def test_span_counts_both_coordinates(oracle_mod, vertical):
    """Reading R5 with the span set by one coordinate alone: a 5-point grid whose neighbours
    lie three auxiliary cells apart in one direction and one cell apart in the other
    (explicit box [0,1]^2, 2^5 cells per side). The span is 3 whichever direction carries it,
    so m = 4 (16 colours), and no two coupled unknowns share a colour."""
    M, L = 8, 5
    prob = five_point_grid(M)
    i = np.arange(M * M) % M
    j = np.arange(M * M) // M
    near, far = (i + 0.5) / 2 ** L, (3 * j + 0.5) / 2 ** L
    x, y = (near, far) if vertical else (far, near)
    h = oracle_mod.Hierarchy(prob.rowptr, prob.col, prob.val, x, y, aux_level=L,
                             bbox=(0.0, 1.0, 0.0, 1.0), coarsest_max=4)
    lv = h.level(0)
    assert lv.span == 3 and lv.m == 4
    np.testing.assert_array_equal(lv.color, lv.t1 % 4 + 4 * (lv.t2 % 4))
    rows = np.repeat(np.arange(lv.n), np.diff(lv.rowptr))
    off = rows != lv.col
    assert np.all(lv.color[rows][off] != lv.color[lv.col][off])


def test_uniform_span_one_gives_four_colours(oracle_mod):
    prob = p1_poisson(33)  # unjittered: aggregation on 2x2 cells of the 31x31 interior nodes
    h = oracle_mod.Hierarchy.from_problem(prob, aux_level=4, coarsest_max=16)
    for l in range(h.nlev):
        lv = h.level(l)
        assert lv.span <= 1 and lv.m == 2 and lv.color.max() <= 3


@pytest.mark.parametrize("case", CASES)
def test_sweeps_are_triangular_solves(oracle_mod, case):
    prob = p1_poisson(**case)
    h = oracle_mod.Hierarchy.from_problem(prob, coarsest_max=4)
    rng = np.random.default_rng(1)
    for l in range(h.nlev - 1):
        lv = h.level(l)
        A = lv.to_scipy().toarray()
        pi = lv.perm
        Ap = A[np.ix_(pi, pi)]
        f = rng.standard_normal(lv.n)
        # forward sweep from zero
        u = h.smooth(l, f, np.zeros(lv.n))
        ref = np.empty(lv.n)
        ref[pi] = sla.solve_triangular(np.tril(Ap), f[pi], lower=True)
        np.testing.assert_allclose(u, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
        # backward sweep from u2
        u2 = rng.standard_normal(lv.n)
        ub = h.smooth(l, f, u2, backward=True)
        ref = u2.copy()
        ref[pi] += sla.solve_triangular(np.triu(Ap), (f - A @ u2)[pi], lower=False)
        np.testing.assert_allclose(ub, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
