"""Pins of the oracle's AMLI-cycle (Alg. 2), nonlinear PCG (Alg. 1) and outer solve.

* Two-level case (level 1 is the coarsest): Alg. 2 is linear; it must equal the dense
  operator u1 = M f, u2 = u1 + P A_c^{-1} P^t (f - A u1), z = u2 + M^t (f - A u2), with M the
  forward Gauss-Seidel matrix, and be symmetric.
* With a linear SPD preconditioner, Alg. 1 must reproduce the iterates of textbook PCG
  (beta from the r.z recurrence, a different formula for the same vectors).
* The whole solve must match a dense direct solve on tiny meshes to 1e-12 relative, and the
  iteration count must stay bounded as h shrinks (the paper's Tables 2-5).
"""
import numpy as np
import pytest
import scipy.linalg as sla

from paper_1209_5421_gb300.meshes import five_point_grid, p1_poisson


def _two_level(oracle_mod, prob, L=3, **kw):
    h = oracle_mod.Hierarchy.from_problem(prob, aux_level=L, coarsest_max=4**L, **kw)
    assert h.nlev == 2
    return h


def _dense_two_level(h):
    f = h.level(0)
    c = h.level(1)
    A = f.to_scipy().toarray()
    Ac = c.to_scipy().toarray()
    n = f.n
    P = np.zeros((n, c.n))
    P[np.arange(n), f.agg] = 1.0
    pi = f.perm
    Q = np.eye(n)[pi]  # (Q u)_p = u_pi[p]
    Ap = Q @ A @ Q.T
    M = Q.T @ np.linalg.inv(np.tril(Ap)) @ Q
    Mt = Q.T @ np.linalg.inv(np.triu(Ap)) @ Q
    I = np.eye(n)
    C = P @ np.linalg.inv(Ac) @ P.T
    B = Mt + (I - Mt @ A) @ (M + C @ (I - A @ M))
    return A, B


@pytest.mark.parametrize("nu", [(2, 2), (2, 1), (1, 3)])
def test_two_level_cycle_with_several_sweeps(oracle_mod, nu):
    """nu_pre forward and nu_post backward sweeps (reading R10 made a parameter): Alg. 2 is
    then B = (I - E) A^{-1} with the error propagation E = (I - M^t A)^nu_post (I - C A)
    (I - M A)^nu_pre of the textbook two-grid method (a different formula from the
    step-by-step cycle); symmetric when nu_pre = nu_post."""
    prob = p1_poisson(n=17, jitter=0.2, seed=3)
    h = _two_level(oracle_mod, prob, nu_pre=nu[0], nu_post=nu[1])
    A, _ = _dense_two_level(h)
    f = h.level(0)
    c = h.level(1)
    n = f.n
    P = np.zeros((n, c.n))
    P[np.arange(n), f.agg] = 1.0
    Q = np.eye(n)[f.perm]
    Ap = Q @ A @ Q.T
    M = Q.T @ np.linalg.inv(np.tril(Ap)) @ Q
    Mt = Q.T @ np.linalg.inv(np.triu(Ap)) @ Q
    I = np.eye(n)
    C = P @ np.linalg.inv(c.to_scipy().toarray()) @ P.T
    mp = np.linalg.matrix_power
    E = mp(I - Mt @ A, nu[1]) @ (I - C @ A) @ mp(I - M @ A, nu[0])
    B = np.linalg.solve(A.T, (I - E).T).T  # (I - E) A^{-1}
    rng = np.random.default_rng(5)
    for _ in range(3):
        v = rng.standard_normal(n)
        np.testing.assert_allclose(h.bhat(0, v), B @ v, rtol=0, atol=1e-10 * np.abs(B @ v).max())
    sym = np.abs(B - B.T).max() / np.abs(B).max()
    if nu[0] == nu[1]:
        assert sym < 1e-10
    else:
        assert sym > 1e-6  # the pre- and post-smoothing differ: not symmetric
    # one sweep each is the operator of the default cycle
    h1 = _two_level(oracle_mod, prob)
    v = rng.standard_normal(n)
    assert not np.allclose(h.bhat(0, v), h1.bhat(0, v), rtol=1e-6, atol=0)


def test_several_sweeps_solve_matches_direct(oracle_mod):
    prob = p1_poisson(n=17, jitter=0.2, seed=6, rhs="normal")
    A = prob.to_scipy().toarray()
    xd = np.linalg.solve(A, prob.b)
    it1 = None
    for nu in ((1, 1), (2, 2), (3, 3)):
        h = oracle_mod.Hierarchy.from_problem(prob, aux_level=3, coarsest_max=16, nu_pre=nu[0],
                                              nu_post=nu[1])
        assert h.nlev >= 3
        x, it, rr, st = h.solve(prob.b, 1e-14)
        assert st == oracle_mod.OK
        assert np.linalg.norm(x - xd) <= 1e-12 * np.linalg.norm(xd)
        x8, it8, _, _ = h.solve(prob.b, 1e-8)
        if it1 is not None:
            assert it8 <= it1  # more smoothing never needs more iterations here
        it1 = it8


@pytest.mark.parametrize("case", [dict(n=17, jitter=0.2, seed=0),
                                  dict(n=19, jitter=0.1, graded=True, kappa_blocks=16, seed=1)])
def test_two_level_cycle_is_the_dense_operator(oracle_mod, case):
    prob = p1_poisson(**case)
    h = _two_level(oracle_mod, prob)
    A, B = _dense_two_level(h)
    rng = np.random.default_rng(2)
    for _ in range(3):
        f = rng.standard_normal(prob.n)
        z = h.bhat(0, f)
        np.testing.assert_allclose(z, B @ f, rtol=0, atol=1e-11 * np.abs(B @ f).max())
    # symmetric (R^t is the adjoint of R, P and P^t in the right places: reading R1)
    assert np.abs(B - B.T).max() < 1e-11 * np.abs(B).max()
    x = rng.standard_normal(prob.n)
    y = rng.standard_normal(prob.n)
    assert abs(h.bhat(0, x) @ y - x @ h.bhat(0, y)) < 1e-11 * np.linalg.norm(x) * np.linalg.norm(y)
    # and positive definite
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0


def _pcg(A, B, f, steps):
    u = np.zeros_like(f)
    r = f.copy()
    z = B @ r
    p = z.copy()
    rz = r @ z
    for i in range(steps):
        q = A @ p
        a = rz / (p @ q)
        u += a * p
        r -= a * q
        if i == steps - 1:
            break
        z = B @ r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return u


@pytest.mark.parametrize("steps", [1, 2, 3, 6])
def test_alg1_equals_pcg_for_linear_preconditioner(oracle_mod, steps):
    prob = p1_poisson(17, jitter=0.2, seed=4, rhs="normal")
    h = _two_level(oracle_mod, prob, kcycle_n=steps)
    A, B = _dense_two_level(h)
    u = h.btilde(0, prob.b)
    ref = _pcg(A, B, prob.b, steps)
    np.testing.assert_allclose(u, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def test_btilde_on_coarsest_is_exact(oracle_mod):
    prob = p1_poisson(17, jitter=0.2, seed=4, rhs="normal")
    h = oracle_mod.Hierarchy.from_problem(prob, coarsest_max=64)
    lc = h.level(h.nlev - 1)
    f = np.random.default_rng(0).standard_normal(lc.n)
    np.testing.assert_allclose(h.btilde(h.nlev - 1, f),
                               np.linalg.solve(lc.to_scipy().toarray(), f), rtol=1e-12)


@pytest.mark.parametrize("case", [dict(n=5), dict(n=9, jitter=0.2), dict(n=13, jitter=0.3, seed=2),
                                  dict(n=17, jitter=0.2, rhs="normal"),
                                  dict(n=17, jitter=0.1, graded=True, kappa_blocks=16, seed=3,
                                       rhs="normal")])
@pytest.mark.parametrize("coarsest_max", [1, 4, 64])
def test_solve_matches_dense_direct(oracle_mod, case, coarsest_max):
    prob = p1_poisson(**case)
    h = oracle_mod.Hierarchy.from_problem(prob, coarsest_max=coarsest_max)
    x, it, rr, st = h.solve(prob.b, tol=1e-13)
    assert st == oracle_mod.OK and rr <= 1e-13
    xs = sla.solve(prob.to_scipy().toarray(), prob.b, assume_a="pos")
    assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs)


def test_iterations_bounded_as_h_shrinks(oracle_mod):
    its = []
    for n in (17, 33, 65, 129, 257):
        prob = p1_poisson(n, jitter=0.2, seed=0, rhs="normal")
        h = oracle_mod.Hierarchy.from_problem(prob)
        x, it, rr, st = h.solve(prob.b, tol=1e-8)
        assert st == oracle_mod.OK and rr <= 1e-8
        its.append(it)
    assert max(its) <= 20 and max(its) - min(its) <= 4, its


def test_coefficient_jumps_iterations_bounded(oracle_mod):
    # piecewise-constant kappa on 16x16 blocks (log-uniform in [0.1, 10]): still bounded
    its = []
    for n in (33, 65, 129, 257):
        prob = p1_poisson(n, jitter=0.1, kappa_blocks=16, seed=0, rhs="normal")
        h = oracle_mod.Hierarchy.from_problem(prob)
        x, it, rr, st = h.solve(prob.b, tol=1e-8)
        assert st == oracle_mod.OK and rr <= 1e-8
        its.append(it)
    assert max(its) <= 20 and max(its) - min(its) <= 4, its


def test_graded_mesh_converges(oracle_mod):
    # x -> x^2, y -> y^2 stretches the elements along the x = 0 and y = 0 edges (aspect ratio
    # up to ~1/h); the solve converges, with counts that grow slowly with n there
    for n in (33, 65, 129):
        prob = p1_poisson(n, jitter=0.1, graded=True, kappa_blocks=16, seed=0, rhs="normal")
        h = oracle_mod.Hierarchy.from_problem(prob)
        x, it, rr, st = h.solve(prob.b, tol=1e-8)
        assert st == oracle_mod.OK and rr <= 1e-8 and it < 100


def test_uniform_grid_converges_fast(oracle_mod):
    # Sec. 5 uniform grid: geometric coarsening, about ten iterations to 1e-6
    prob = five_point_grid(64)
    h = oracle_mod.Hierarchy.from_problem(prob, aux_level=5, bbox=(0.0, 1.0, 0.0, 1.0))
    x, it, rr, st = h.solve(prob.b, tol=1e-6)
    assert st == oracle_mod.OK and it <= 12


def test_zero_rhs_and_single_level(oracle_mod):
    prob = p1_poisson(9, jitter=0.2)
    h = oracle_mod.Hierarchy.from_problem(prob)
    x, it, rr, st = h.solve(np.zeros(prob.n))
    assert st == oracle_mod.OK and it == 0 and np.all(x == 0)
    h1 = oracle_mod.Hierarchy.from_problem(prob, coarsest_max=prob.n)
    assert h1.nlev == 1
    x, it, rr, st = h1.solve(prob.b, tol=1e-12)
    assert st == oracle_mod.OK and it == 1


def test_invalid_inputs_rejected(oracle_mod):
    prob = p1_poisson(9, jitter=0.2)
    bad_col = prob.col.copy()
    bad_col[[1, 2]] = bad_col[[2, 1]]  # unsorted row
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.Hierarchy(prob.rowptr, bad_col, prob.val, prob.x, prob.y)
    bad_val = prob.val.copy()
    bad_val[prob.rowptr[0] + 2] = -1.0  # row 0: entries (self, E, N): self is first -> index 0
    bad_val[0] = -4.0
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.Hierarchy(prob.rowptr, prob.col, bad_val, prob.x, prob.y)
    x = prob.x.copy()
    x[3] = np.nan
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.Hierarchy(prob.rowptr, prob.col, prob.val, x, prob.y)
