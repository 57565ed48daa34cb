"""Pins of the oracle's Galerkin coarse operators (Sec. 2 eqs. def:Ac / acsum, Sec. 4.4).

Checked against: an explicit sparse triple product P^t A P with P built as the Boolean
matrix of eq. def:P (scipy, a textbook product); symmetry; A 1 = 0 preserved in the pure
Neumann case; and the closed form on the uniform grid (Sec. 5), where level k of the 5-point
Laplacian is 2^(L+1-k) times the 5-point stencil.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_1209_5421_gb300.meshes import five_point_grid, p1_poisson


def _P(agg, nc):
    n = len(agg)
    return sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, nc))


CASES = [
    dict(n=33, jitter=0.2, seed=0),
    dict(n=41, jitter=0.1, graded=True, kappa_blocks=16, seed=2),
    dict(n=29, jitter=0.3, seed=5),
]


@pytest.mark.parametrize("case", CASES)
def test_galerkin_equals_triple_product(oracle_mod, case):
    prob = p1_poisson(**case)
    h = oracle_mod.Hierarchy.from_problem(prob, coarsest_max=4)
    assert h.nlev >= 3
    for l in range(h.nlev - 1):
        f = h.level(l)
        c = h.level(l + 1)
        P = _P(f.agg, c.n)
        ref = (P.T @ f.to_scipy() @ P).toarray()
        got = c.to_scipy().toarray()
        scale = np.abs(ref).max()
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14 * scale)
        # stored pattern = the pairs (R, C) that receive a contribution
        pat = (abs(P.T) @ abs(f.to_scipy()).sign() @ P).toarray() != 0
        np.testing.assert_array_equal(c.to_scipy().toarray() != 0, pat & (got != 0))
        assert (c.to_scipy() != 0).sum() <= pat.sum()


@pytest.mark.parametrize("case", CASES + [dict(n=33, jitter=0.0, seed=0)])
def test_stored_pattern_is_every_contributed_pair(oracle_mod, case):
    """Readings R6 / R7 / R17: a coarse operator stores every pair (R, C) that receives a
    contribution of eq. acsum, also when the sum is exactly zero. The expected structure is
    that of P^t S P, with S holding a one for every stored fine entry (a sum of ones cannot
    cancel). The unjittered mesh has exactly-zero couplings on its diagonal edges, so there
    the coarse levels store exact zeros."""
    prob = p1_poisson(**case)
    h = oracle_mod.Hierarchy.from_problem(prob, coarsest_max=4)
    zeros = 0
    for l in range(h.nlev - 1):
        f = h.level(l)
        c = h.level(l + 1)
        P = _P(f.agg, c.n)
        S = sp.csr_matrix((np.ones(len(f.col)), f.col, f.rowptr), shape=(f.n, f.n))
        E = (P.T @ S @ P).tocsr()
        E.sort_indices()
        np.testing.assert_array_equal(c.rowptr, E.indptr)
        np.testing.assert_array_equal(c.col, E.indices)
        zeros += int((c.val == 0.0).sum())
    if case["jitter"] == 0.0:
        assert zeros > 0


@pytest.mark.parametrize("case", CASES)
def test_coarse_operators_symmetric(oracle_mod, case):
    prob = p1_poisson(**case)
    h = oracle_mod.Hierarchy.from_problem(prob, coarsest_max=4)
    for l in range(1, h.nlev):
        A = h.level(l).to_scipy().toarray()
        assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()


def test_neumann_constants_preserved(oracle_mod):
    # pure Neumann: A 1 = 0  =>  P^t A P 1 = P^t A 1 = 0 on every level
    prob = p1_poisson(33, jitter=0.2, dirichlet=False, seed=4)
    A = prob.to_scipy()
    assert np.abs(A @ np.ones(prob.n)).max() < 1e-13 * abs(A).max()
    h = oracle_mod.Hierarchy.from_problem(prob, coarsest_max=1, no_factor=True)
    assert h.nlev >= 5
    # rounding scale of each coarse row: the sum of |a_ij| over the fine entries it collects
    absrow = np.asarray(abs(A).sum(axis=1)).ravel()
    for l in range(1, h.nlev):
        lv = h.level(l)
        absrow = np.bincount(h.level(l - 1).agg, weights=absrow, minlength=lv.n)
        Ak = lv.to_scipy()
        assert np.all(np.abs(Ak @ np.ones(lv.n)) <= 1e-14 * absrow), l
        # and the level really carries the operator: entries are not all rounding noise
        assert abs(Ak).max() > 1e-3 * absrow.max() or lv.n == 1


def test_uniform_grid_closed_form(oracle_mod):
    L = 5
    M = 2 ** (L + 1)
    prob = five_point_grid(M)
    h = oracle_mod.Hierarchy.from_problem(prob, aux_level=L, bbox=(0.0, 1.0, 0.0, 1.0),
                                          coarsest_max=16)
    for l in range(1, h.nlev):
        lv = h.level(l)
        k = L - (l - 1)
        W = 2**k
        A = lv.to_scipy().tocsr()
        c = 2 ** (L + 1 - k)
        for R in range(lv.n):
            t1, t2 = R % W, R // W
            if t1 in (0, W - 1) or t2 in (0, W - 1):
                continue
            cols = A.indices[A.indptr[R]:A.indptr[R + 1]]
            vals = A.data[A.indptr[R]:A.indptr[R + 1]]
            row = dict(zip(cols.tolist(), vals.tolist()))
            # interior rows: c * [4, -1, -1, -1, -1]; no diagonal neighbours (Sec. 4.4 pattern)
            assert row == {R: 4.0 * c, R - 1: -c, R + 1: -c, R - W: -c, R + W: -c}, (l, R)
        # the span is one cell, so four colours (Sec. 4.5)
        assert lv.span == 1 and lv.m == 2
