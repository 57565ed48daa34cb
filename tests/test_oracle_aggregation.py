"""Pins of the oracle's auxiliary-grid aggregation (Sec. 3.1, 3.2, 4.2, 4.3 of the paper).

Each check uses arithmetic other than the oracle's: exact rational binning against the boxes
of eq. subregion, the closed-form 2x2 blocks of the uniform grid (Sec. 5), the explicit
four-child restriction formula (Sec. 4.3), the coarse-level parent listing form (Sec. 4.2).
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_1209_5421_gb300.meshes import five_point_grid, p1_poisson


def test_auto_level_is_floor_log4(oracle_mod):
    # Sec. 3.1: L = floor(log N / log 4), i.e. 4^L <= N < 4^(L+1)
    for N in list(range(1, 300)) + [4**k for k in range(1, 15)] + [4**k - 1 for k in range(2, 15)] \
            + [1046529, 2093809, 3969]:
        L = oracle_mod.auto_level(N)
        assert 4**L <= N < 4 ** (L + 1), (N, L)
    assert oracle_mod.auto_level(2093809) == 10
    assert oracle_mod.auto_level(1046529) == 9


def _exact_cell(v, lo, hi, L):
    """Cell of v among the 2^L boxes of eq. subregion, in exact rational arithmetic.
    Boxes are half-open [lo + t w, lo + (t+1) w) except the last, which is closed."""
    w = 2**L
    q = (Fraction(v) - Fraction(lo)) * w / (Fraction(hi) - Fraction(lo))
    t = int(q // 1)
    return min(max(t, 0), w - 1), q


@pytest.mark.parametrize("L", [1, 3, 6])
def test_binning_matches_exact_boxes(oracle_mod, L):
    prob = p1_poisson(33, jitter=0.2, seed=3)
    rng = np.random.default_rng(7)
    x = np.concatenate([prob.x, rng.uniform(0, 1, 500)])
    y = np.concatenate([prob.y, rng.uniform(0, 1, 500)])
    bbox = np.array([x.min(), x.max(), y.min(), y.max()])
    cell = oracle_mod.bin_points(x, y, bbox, L)
    w = 2**L
    near = 0
    for j in range(len(x)):
        tx, qx = _exact_cell(x[j], bbox[0], bbox[1], L)
        ty, qy = _exact_cell(y[j], bbox[2], bbox[3], L)
        if cell[j] != ty * w + tx:
            # only a point within rounding of a box edge may land in the neighbouring box
            dx = abs(float(qx - round(qx)))
            dy = abs(float(qy - round(qy)))
            assert min(dx, dy) < 1e-12, (j, cell[j], ty * w + tx)
            near += 1
    assert near == 0
    # the closed upper edge belongs to the last cell (reading R4)
    assert cell[np.argmax(x)] % w == w - 1
    assert cell[np.argmax(y)] // w == w - 1


def test_setup_box_is_each_coordinates_extent(oracle_mod):
    """Sec. 3.1 eq. ab12 in the setup path: the auxiliary box is the extent of each coordinate
    separately. On a mesh stretched to x in [0.5, 3.5] and shifted to y in [-2, -1], the box is
    numpy's min / max of each coordinate, and every unknown's level-L cell is its exact eq.
    subregion box within that extent."""
    prob = p1_poisson(33, jitter=0.2, seed=4)
    x, y = 3.0 * prob.x + 0.5, prob.y - 2.0
    L = 4
    h = oracle_mod.Hierarchy(prob.rowptr, prob.col, prob.val, x, y, aux_level=L,
                             coarsest_max=16)
    np.testing.assert_array_equal(h.bbox, [x.min(), x.max(), y.min(), y.max()])
    lv = h.level(0)
    for j in range(len(x)):
        assert lv.t1[j] == _exact_cell(x[j], x.min(), x.max(), L)[0], j
        assert lv.t2[j] == _exact_cell(y[j], y.min(), y.max(), L)[0], j


def test_uniform_grid_aggregates_are_2x2_blocks(oracle_mod):
    # Sec. 5 (uniform grid): aggregation coincides with geometric coarsening
    L = 4
    M = 2 ** (L + 1)
    prob = five_point_grid(M)
    h = oracle_mod.Hierarchy.from_problem(prob, aux_level=L, bbox=(0.0, 1.0, 0.0, 1.0),
                                          coarsest_max=4)
    fine = h.level(0)
    i = np.arange(prob.n) % M
    j = np.arange(prob.n) // M
    np.testing.assert_array_equal(fine.agg, (j // 2) * 2**L + (i // 2))
    # every coarse level is the full 2^k x 2^k grid, rows in lexicographic cell order
    for l in range(1, h.nlev):
        lv = h.level(l)
        k = L - (l - 1)
        assert lv.n == 4**k and lv.cellw == 2**k
        np.testing.assert_array_equal(lv.t1 + 2**k * lv.t2, np.arange(lv.n))


def test_coarse_parent_listing_and_restriction_formula(oracle_mod):
    # Sec. 4.2 coarse-level listing: child j at width W has parent ((j/W)/2)*(W/2) + (j%W)/2.
    # Sec. 4.3: (v^{k-1})_i = v_{2t1+2^k(2t2)} + v_{2t1+1+2^k(2t2)} + v_{2t1+1+2^k(2t2+1)}
    #                         + v_{2t1+2^k(2t2+1)},  i = t1 + 2^{k-1} t2.
    L = 5
    prob = five_point_grid(2 ** (L + 1))
    h = oracle_mod.Hierarchy.from_problem(prob, aux_level=L, bbox=(0.0, 1.0, 0.0, 1.0),
                                          coarsest_max=1)
    rng = np.random.default_rng(0)
    for l in range(1, h.nlev - 1):
        lv = h.level(l)
        W = lv.cellw
        jidx = np.arange(lv.n)
        np.testing.assert_array_equal(lv.agg, ((jidx // W) // 2) * (W // 2) + (jidx % W) // 2)
        v = rng.standard_normal(lv.n)
        restricted = np.zeros(h.level(l + 1).n)
        np.add.at(restricted, lv.agg, v)  # P^t v from the oracle's aggregates
        Wc = W // 2
        t1, t2 = np.meshgrid(np.arange(Wc), np.arange(Wc), indexing="xy")
        t1, t2 = t1.ravel(), t2.ravel()
        explicit = (v[2 * t1 + W * (2 * t2)] + v[2 * t1 + 1 + W * (2 * t2)]
                    + v[(2 * t1 + 1) + W * (2 * t2 + 1)] + v[2 * t1 + W * (2 * t2 + 1)])
        np.testing.assert_allclose(restricted[t1 + Wc * t2], explicit, rtol=0, atol=1e-13)


def test_empty_cells_are_compacted_in_cell_order(oracle_mod):
    # aggregates must be non-empty (Sec. 2); empty auxiliary cells occur (Sec. 5, disk domain)
    prob = p1_poisson(41, jitter=0.1, graded=True, seed=1)
    L = 5
    h = oracle_mod.Hierarchy.from_problem(prob, aux_level=L, coarsest_max=8)
    fine = h.level(0)
    cells = fine.t2 * 2**L + fine.t1
    occupied = np.unique(cells)
    assert len(occupied) < 4**L  # the graded mesh leaves cells empty
    np.testing.assert_array_equal(fine.agg, np.searchsorted(occupied, cells))
    for l in range(1, h.nlev - 1):
        lv = h.level(l)
        parent = (lv.t2 >> 1) * (lv.cellw // 2) + (lv.t1 >> 1)
        occ = np.unique(parent)
        np.testing.assert_array_equal(lv.agg, np.searchsorted(occ, parent))
        nxt = h.level(l + 1)
        np.testing.assert_array_equal(nxt.t1 + nxt.cellw * nxt.t2, occ)
        assert np.bincount(lv.agg, minlength=nxt.n).min() >= 1


def test_depth_and_coarsest_level(oracle_mod):
    prob = p1_poisson(65, jitter=0.2)
    h = oracle_mod.Hierarchy.from_problem(prob, aux_level=6, coarsest_max=64)
    sizes = [h.level(l).n for l in range(h.nlev)]
    assert sizes[-1] <= 64 and all(s > 64 for s in sizes[:-1])
    assert h.level(1).cellw == 64 and h.level(h.nlev - 1).cellw == 8
    # a problem no larger than coarsest_max is solved directly on one level
    small = p1_poisson(6)
    hs = oracle_mod.Hierarchy.from_problem(small, coarsest_max=64)
    assert hs.nlev == 1
