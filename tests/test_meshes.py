"""Self-checks of the seeded synthetic workloads (input generation, not the method)."""
import numpy as np
import pytest

from paper_1209_5421_gb300.meshes import five_point_grid, p1_poisson, workload


def test_uniform_p1_mesh_is_five_point_stencil():
    # Sec. 5: on a uniform grid linear finite elements give the 5-point stencil
    prob = p1_poisson(9)
    A = prob.to_scipy().toarray()
    m = 7
    for k in range(prob.n):
        i, j = k % m, k // m
        ref = np.zeros(prob.n)
        ref[k] = 4.0
        for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            if 0 <= i + di < m and 0 <= j + dj < m:
                ref[(j + dj) * m + i + di] = -1.0
        np.testing.assert_array_equal(A[k], ref)
    # pattern keeps the 7-point couplings of the triangulation (explicit zeros on diagonals)
    assert prob.nnz == m * m + 4 * m * (m - 1) + 2 * (m - 1) ** 2


@pytest.mark.parametrize("kw", [dict(jitter=0.2), dict(jitter=0.1, graded=True, kappa_blocks=16)])
def test_spd_symmetric_and_neumann_kernel(kw):
    prob = p1_poisson(21, seed=3, **kw)
    A = prob.to_scipy()
    assert abs(A - A.T).max() == 0.0
    assert np.linalg.eigvalsh(A.toarray()).min() > 0
    neu = p1_poisson(21, seed=3, dirichlet=False, **kw).to_scipy()
    assert np.abs(neu @ np.ones(neu.shape[0])).max() < 1e-13 * abs(neu).max()
    # columns sorted and unique, diagonal present
    for i in range(prob.n):
        c = prob.col[prob.rowptr[i]:prob.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0) and i in c


def test_seeded_and_deterministic():
    a = p1_poisson(33, jitter=0.2, seed=5, rhs="normal")
    b = p1_poisson(33, jitter=0.2, seed=5, rhs="normal")
    c = p1_poisson(33, jitter=0.2, seed=6, rhs="normal")
    assert np.array_equal(a.val, b.val) and np.array_equal(a.b, b.b)
    assert not np.array_equal(a.x, c.x)
    # jitter bounded by 0.2 h around the lattice
    h = 1 / 32
    lattice = (np.arange(a.n) % 31 + 1) * h
    assert np.abs(a.x - lattice).max() <= 0.2 * h


def test_load_vector_integrates_f_equal_one():
    # Neumann load vector of f = 1 sums to the area of the unit square
    prob = p1_poisson(17, jitter=0.2, dirichlet=False)
    assert abs(prob.b.sum() - 1.0) < 1e-14


def test_named_workload_sizes():
    p, L = workload("quasi_uniform_65")
    assert (p.n, L) == (63 * 63, 6)
    p = five_point_grid(8)
    assert p.n == 64 and p.nnz == 64 * 5 - 4 * 8
