"""Pins of the oracle on the disk domain (the paper's Sec. 5 disk examples): the auxiliary
grid over the nodes' bounding box has empty cells in its corners, and the method must still
build non-empty aggregates (compacted in cell order), exact Galerkin operators and converge.

Checked against: brute-force occupancy of the level-L cells recomputed here from the
oracle's own cell coordinates; scipy's P^t A P; the dense direct solve (1e-12); and the
iteration count of the same mesh on the full square (the disk must not be harder).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_1209_5421_gb300.meshes import disk_poisson, p1_poisson


def test_disk_mesh_is_spd_submatrix():
    sq = p1_poisson(33, jitter=0.2, seed=4, rhs="zero")
    dk = disk_poisson(33, jitter=0.2, seed=4)
    keep = np.flatnonzero((sq.x - 0.5) ** 2 + (sq.y - 0.5) ** 2 < 0.25)
    A = sq.to_scipy()[keep][:, keep].toarray()
    np.testing.assert_array_equal(dk.to_scipy().toarray(), A)
    assert np.linalg.eigvalsh(A).min() > 0
    np.testing.assert_array_equal(dk.x, sq.x[keep])


@pytest.mark.parametrize("n,L", [(65, 6), (49, 5)])
def test_disk_aggregates_skip_empty_cells(oracle_mod, n, L):
    prob = disk_poisson(n, seed=1)
    h = oracle_mod.Hierarchy.from_problem(prob, aux_level=L, coarsest_max=16)
    fine = h.level(0)
    cells = fine.t2 * 2**L + fine.t1
    occupied = np.unique(cells)
    assert len(occupied) < 0.85 * 4**L  # the corners outside the disk are empty
    np.testing.assert_array_equal(fine.agg, np.searchsorted(occupied, cells))
    assert h.level(1).n == len(occupied)
    for l in range(1, h.nlev - 1):
        lv, nxt = h.level(l), h.level(l + 1)
        parent = (lv.t2 >> 1) * (lv.cellw // 2) + (lv.t1 >> 1)
        occ = np.unique(parent)
        np.testing.assert_array_equal(lv.agg, np.searchsorted(occ, parent))
        assert nxt.n == len(occ)
        assert np.bincount(lv.agg, minlength=nxt.n).min() >= 1
        P = sp.csr_matrix((np.ones(lv.n), (np.arange(lv.n), lv.agg)), shape=(lv.n, nxt.n))
        ref = (P.T @ lv.to_scipy() @ P).toarray()
        np.testing.assert_allclose(nxt.to_scipy().toarray(), ref, rtol=0,
                                   atol=1e-14 * np.abs(ref).max())


def test_disk_solve_matches_dense_and_is_not_harder(oracle_mod):
    prob = disk_poisson(65, seed=3)
    h = oracle_mod.Hierarchy.from_problem(prob)
    x, it, rr, st = h.solve(prob.b, 1e-12)
    assert st == oracle_mod.OK
    xd = np.linalg.solve(prob.to_scipy().toarray(), prob.b)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    sq = p1_poisson(65, jitter=0.2, seed=3, rhs="normal")
    _, it_sq, _, _ = oracle_mod.Hierarchy.from_problem(sq).solve(sq.b, 1e-12)
    assert it <= it_sq + 2, (it, it_sq)
