"""Pins of the oracle's octree (3D) variant of the auxiliary-grid aggregation (Sec. 3.1: the
same construction with 8 children per cell; Sec. 6: 27-point coarse stencils, 8 colours).

Checked against: exact rational binning into the boxes of eq. subregion in three
coordinates; the octree depth rule 8^L <= N; brute-force occupancy and the listing form of
the parent (every coordinate halved); scipy's P^t A P; the colouring's defining property (no
two coupled rows share a colour); the dense direct solve; bounded iteration counts as h
shrinks; and the tetrahedral mesh itself (symmetric, positive definite, Kuhn topology).
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1209_5421_gb300.meshes import p1_poisson_3d


def _exact_cell(v, lo, hi, L):
    w = 2**L
    q = (Fraction(v) - Fraction(lo)) * w / (Fraction(hi) - Fraction(lo))
    return min(max(int(q // 1), 0), w - 1)


def test_mesh_is_spd_kuhn():
    p = p1_poisson_3d(6, seed=2)
    A = p.to_scipy().toarray()
    assert np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0
    # Kuhn topology: interior rows couple to themselves and 14 neighbours (15-point)
    assert np.diff(p.rowptr).max() == 15
    # without jitter the off-diagonal couplings are those of the 15-point stencil only
    q = p1_poisson_3d(6, jitter=0.0, seed=0)
    i = 2 + 4 * (2 + 4 * 2)  # an interior unknown (4^3 unknowns, x fastest)
    cols = q.col[q.rowptr[i]:q.rowptr[i + 1]]
    d = set()
    for j in cols:
        dx, dy, dz = j % 4 - i % 4, (j // 4) % 4 - (i // 4) % 4, j // 16 - i // 16
        d.add((dx, dy, dz))
    expect = {(0, 0, 0)}
    for v in [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]:
        expect.add(v)
        expect.add(tuple(-c for c in v))
    assert d == expect


def test_octree_depth_rule(oracle_mod):
    for N in list(range(1, 600)) + [8**k for k in range(1, 10)] + [8**k - 1 for k in range(2, 10)]:
        L = oracle_mod.auto_level(N, dim=3)
        assert 8**L <= N < 8 ** (L + 1), (N, L)


@pytest.mark.parametrize("L", [1, 3, 5])
def test_octree_binning_matches_exact_boxes(oracle_mod, L):
    p = p1_poisson_3d(9, seed=3)
    rng = np.random.default_rng(L)
    x = np.concatenate([p.x, rng.uniform(0, 1, 300)])
    y = np.concatenate([p.y, rng.uniform(0, 1, 300)])
    z = np.concatenate([p.z, rng.uniform(0, 1, 300)])
    bb = np.array([x.min(), x.max(), y.min(), y.max(), z.min(), z.max()])
    cell = oracle_mod.bin_points3(x, y, z, bb, L)
    w = 2**L
    for j in range(len(x)):
        t = [_exact_cell(v, bb[2 * d], bb[2 * d + 1], L) for d, v in enumerate((x[j], y[j], z[j]))]
        assert cell[j] == t[0] + w * t[1] + w * w * t[2], j
    assert cell[np.argmax(z)] // (w * w) == w - 1  # the closed upper face belongs to the last cell


def test_octree_setup_box_is_each_coordinates_extent(oracle_mod):
    """Sec. 3.1 eq. ab12 in three coordinates, in the setup path: on a mesh whose coordinates
    have three different extents (x in [0, 1], y in [1, 3], z in [-1, 2]) the box is numpy's
    min / max of each coordinate, and every unknown's level-L cell is its exact eq. subregion
    box within those extents."""
    p = p1_poisson_3d(9, seed=5)
    x, y, z = p.x, 2.0 * p.y + 1.0, 3.0 * p.z - 1.0
    L = 2
    h = oracle_mod.Hierarchy(p.rowptr, p.col, p.val, x, y, z=z, aux_level=L, coarsest_max=8)
    np.testing.assert_array_equal(h.bbox, [x.min(), x.max(), y.min(), y.max()])
    np.testing.assert_array_equal(h.zbox, [z.min(), z.max()])
    lv = h.level(0)
    for j in range(len(x)):
        t = [_exact_cell(v, lo, hi, L) for v, lo, hi in
             ((x[j], x.min(), x.max()), (y[j], y.min(), y.max()), (z[j], z.min(), z.max()))]
        assert (lv.t1[j], lv.t2[j], lv.t3[j]) == tuple(t), j


@pytest.mark.parametrize("far", [0, 1, 2])
def test_octree_span_counts_every_coordinate(oracle_mod, far):
    """Reading R5 in 3D (R23) with the span set by one coordinate alone: a 7-point grid of 4^3
    unknowns whose neighbours lie three auxiliary cells apart along axis `far` and one cell
    apart along the other two (explicit box [0,1]^3, 2^4 cells per side). The span is 3
    whichever axis carries it, so m = 4 (64 colours), and no two coupled unknowns share a
    colour."""
    M, L = 4, 4
    T = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(M, M))
    I = sp.identity(M)
    A = (sp.kron(sp.kron(I, I), T) + sp.kron(sp.kron(I, T), I) + sp.kron(sp.kron(T, I), I)).tocsr()
    A.eliminate_zeros()  # kron stores the zero blocks, and a stored entry is a coupling
    A.sort_indices()
    k = np.arange(M ** 3)
    idx = [k % M, (k // M) % M, k // (M * M)]  # x fastest, as the matrix is ordered
    xyz = [(3 * c + 0.5) / 2 ** L if d == far else (c + 0.5) / 2 ** L for d, c in enumerate(idx)]
    h = oracle_mod.Hierarchy(A.indptr, A.indices, A.data, xyz[0], xyz[1], z=xyz[2], aux_level=L,
                             bbox=(0.0, 1.0, 0.0, 1.0, 0.0, 1.0), coarsest_max=4)
    lv = h.level(0)
    assert lv.span == 3 and lv.m == 4
    np.testing.assert_array_equal(lv.color, lv.t1 % 4 + 4 * (lv.t2 % 4) + 16 * (lv.t3 % 4))
    rows = np.repeat(np.arange(lv.n), np.diff(lv.rowptr))
    off = rows != lv.col
    assert np.all(lv.color[rows][off] != lv.color[lv.col][off])


@pytest.mark.parametrize("n", [9, 17])
def test_octree_aggregation_galerkin_colours(oracle_mod, n):
    p = p1_poisson_3d(n, seed=n)
    h = oracle_mod.Hierarchy.from_problem(p, coarsest_max=8)
    assert h.dim == 3 and h.nlev >= 3
    f = h.level(0)
    w = 2**h.L
    cells = f.t1 + w * (f.t2 + w * f.t3)
    occ = np.unique(cells)
    np.testing.assert_array_equal(f.agg, np.searchsorted(occ, cells))
    for l in range(h.nlev - 1):
        lv, nx = h.level(l), h.level(l + 1)
        if l > 0:  # the parent halves every coordinate (listing form, Sec. 4.2, in 3D)
            wc = lv.cellw // 2
            parent = (lv.t1 >> 1) + wc * ((lv.t2 >> 1) + wc * (lv.t3 >> 1))
            occp = np.unique(parent)
            np.testing.assert_array_equal(lv.agg, np.searchsorted(occp, parent))
            np.testing.assert_array_equal(nx.t1 + wc * (nx.t2 + wc * nx.t3), occp)
        counts = np.bincount(lv.agg, minlength=nx.n)
        assert counts.min() >= 1 and (l == 0 or counts.max() <= 8)
        P = sp.csr_matrix((np.ones(lv.n), (np.arange(lv.n), lv.agg)), shape=(lv.n, nx.n))
        ref = (P.T @ lv.to_scipy() @ P).toarray()
        np.testing.assert_allclose(nx.to_scipy().toarray(), ref, rtol=0,
                                   atol=1e-14 * np.abs(ref).max())
    for l in range(1, h.nlev):  # 27-point coarse stencils, m^3 colours, no coupled pair shares one
        lv = h.level(l)
        A = lv.to_scipy().tocoo()
        assert lv.span <= 1 and lv.m == 2
        assert np.diff(lv.rowptr).max() <= 27
        off = A.row != A.col
        assert not np.any(lv.color[A.row[off]] == lv.color[A.col[off]])
        assert set(np.unique(lv.color)) <= set(range(8))


def test_octree_solve_matches_dense_direct(oracle_mod):
    p = p1_poisson_3d(7, seed=5)
    h = oracle_mod.Hierarchy.from_problem(p, coarsest_max=4)
    assert h.nlev >= 2
    x, it, rr, st = h.solve(p.b, 1e-13)
    assert st == oracle_mod.OK
    xd = np.linalg.solve(p.to_scipy().toarray(), p.b)
    assert np.linalg.norm(x - xd) <= 1e-12 * np.linalg.norm(xd)


def test_octree_iterations_bounded(oracle_mod):
    its = []
    for n in (9, 17, 33):
        p = p1_poisson_3d(n, seed=1)
        h = oracle_mod.Hierarchy.from_problem(p)
        _, it, _, st = h.solve(p.b, 1e-8)
        assert st == oracle_mod.OK
        its.append(it)
    assert max(its) <= 20 and its[-1] - its[0] <= 6, its
