"""Pins of the oracle's eigenvalue solve: brute force on explicit Kronecker
matrices, closed forms, KKT invariants, and independent optimisers."""

import numpy as np
import pytest
import scipy.optimize

from oracle import kron
from oracle.solve import (KSProblem, gradient, hessian, objective, rel_kkt,
                          solve_alg1, solve_newton, two_axis_problem)
from oracle.spectra import top_eigh, two_axis_spectra
from synth import planted_c1


def _rand_problem(rng, r1, r2):
    e1 = np.sort(rng.uniform(1.0, 50.0, r1))[::-1]
    e2 = np.sort(rng.uniform(1.0, 50.0, r2))[::-1]
    return two_axis_problem(e1, e2)


def test_kronecker_sum_identity_eigenpairs():
    # Introduction: F (+) G = F (x) I + I (x) G; eigenpairs (f_i + g_j, u_i (x) w_j).
    rng = np.random.default_rng(5)
    a = rng.standard_normal((3, 3)); f = a + a.T
    b = rng.standard_normal((4, 4)); g = b + b.T
    ks = kron.kron_sum(f, g)
    np.testing.assert_allclose(ks, np.kron(f, np.eye(4)) + np.kron(np.eye(3), g))
    lf, uf = np.linalg.eigh(f)
    lg, ug = np.linalg.eigh(g)
    for i in range(3):
        for j in range(4):
            v = np.kron(uf[:, i], ug[:, j])
            np.testing.assert_allclose(ks @ v, (lf[i] + lg[j]) * v, atol=1e-12)


def test_gradient_and_hessian_match_finite_differences():
    rng = np.random.default_rng(6)
    prob = KSProblem([np.sort(rng.uniform(1, 5, n))[::-1] for n in (3, 4, 2)],
                     [(0, 1, 2), (0, 1)])
    x = rng.uniform(0.5, 2.0, prob.n)
    g = gradient(x, prob)
    h = hessian(x, prob)
    step = 1e-6
    for i in range(prob.n):
        e = np.zeros(prob.n); e[i] = step
        fd = (objective(x + e, prob) - objective(x - e, prob)) / (2 * step)
        assert abs(fd - g[i]) <= 1e-6 * (1 + abs(g[i]))
        gd = (gradient(x + e, prob) - gradient(x - e, prob)) / (2 * step)
        np.testing.assert_allclose(gd, h[:, i], rtol=1e-5, atol=1e-7)


def test_objective_equals_dense_singular_likelihood():
    # The grid formula sum E.Lam - sum log(lam_i + mu_j) must equal the
    # -2 log-likelihood computed from explicit d1 d2 x d1 d2 matrices with
    # the pseudo-determinant (appendix on the singular distribution).
    rng = np.random.default_rng(7)
    x = rng.standard_normal((4, 3))
    e_r, v_r = top_eigh(x @ x.T, 2)   # truncated row axis
    e_c, v_c = top_eigh(x.T @ x, 3)
    prob = two_axis_problem(e_r, e_c)
    for _ in range(3):
        lam = rng.uniform(0.2, 2.0, 2)
        mu = rng.uniform(0.2, 2.0, 3)
        f = objective(np.concatenate([lam, mu]), prob)
        dense = kron.dense_nll_singular(x, v_r, lam, v_c, mu)
        assert abs(f - dense) <= 1e-10 * (1 + abs(f))


def test_brute_force_full_rank_mle_matches_eigen_method():
    # Brute force over dense PD Psi_rows = A A^T, Psi_cols = B B^T for four
    # iid 3 x 3 draws: maximise the explicit 9-dim Gaussian likelihood; the
    # Kronecker sum (identifiable) must equal the eigen-method's, where the
    # iid draws enter as modalities sharing both axes (S_l summed, one log-det
    # grid per draw).  Also Theorem 1: the brute-force Psi_l commute with S_l.
    rng = np.random.default_rng(8)
    xs = [rng.standard_normal((3, 3)) for _ in range(4)]
    il = np.tril_indices(3)

    def unpack(th):
        a = np.zeros((3, 3)); a[il] = th[:6]
        b = np.zeros((3, 3)); b[il] = th[6:]
        return a @ a.T, b @ b.T

    def nll(th):
        a, b = unpack(th)
        return sum(kron.dense_nll_full(x, a, b) for x in xs)

    th0 = np.concatenate([np.eye(3)[il], np.eye(3)[il]])
    res = scipy.optimize.minimize(nll, th0, method="BFGS",
                                  options={"gtol": 1e-9, "maxiter": 20000})
    a, b = unpack(res.x)
    brute = kron.kron_sum(b, a)
    s_r = sum(x @ x.T for x in xs)
    s_c = sum(x.T @ x for x in xs)
    e_r, v_r = top_eigh(s_r, 3)
    e_c, v_c = top_eigh(s_c, 3)
    prob = KSProblem([e_r, e_c], [(0, 1)] * 4)
    lam, info = solve_newton(prob)
    assert info.converged
    psi_r = (v_r * lam[:3]) @ v_r.T
    psi_c = (v_c * lam[3:]) @ v_c.T
    ours = kron.kron_sum(psi_c, psi_r)
    np.testing.assert_allclose(ours, brute, atol=1e-4 * np.abs(brute).max())
    np.testing.assert_allclose(a @ s_r, s_r @ a, atol=1e-4 * np.abs(s_r).max() * np.abs(a).max())


def test_brute_force_truncated_matches_eigen_method():
    # Truncated rows (r1 = 2 < 4): minimise the explicit dense pseudo-det
    # likelihood over (lam, mu) with a generic bounded optimiser.
    rng = np.random.default_rng(9)
    x = rng.standard_normal((4, 3))
    e_r, v_r = top_eigh(x @ x.T, 2)
    e_c, v_c = top_eigh(x.T @ x, 3)
    prob = two_axis_problem(e_r, e_c)
    sol, info = solve_newton(prob)
    assert info.converged

    def fun(z):
        return kron.dense_nll_singular(x, v_r, z[:2], v_c, z[2:])

    lo = prob.eps[0]
    res = scipy.optimize.minimize(fun, np.concatenate([1 / e_r, 1 / e_c]), method="L-BFGS-B",
                                  bounds=[(lo, None)] * 5,
                                  options={"ftol": 1e-15, "gtol": 1e-12, "maxiter": 20000})
    s_ours = sol[:2, None] + sol[None, 2:]
    s_brute = res.x[:2, None] + res.x[None, 2:]
    np.testing.assert_allclose(s_ours, s_brute, rtol=2e-4)
    assert fun(sol) <= res.fun + 1e-9 * abs(res.fun)


def _kkt_invariants(prob, x, tol=1e-9):
    g = gradient(x, prob)
    lo = prob.lower()
    at = x <= lo
    e = prob.e_all()
    assert np.all(np.abs(g[~at]) <= tol * e[~at])
    assert np.all(g[at] >= -tol * e[at])
    return g, at


def test_kkt_and_trace_identity_with_truncated_rows():
    # sum of all stationarity equations: sum over bound mu of g - sum over
    # bound lam of g = tr E_cols - tr E_rows.
    x, _, _ = planted_c1()
    e_r, _, e_c, _ = two_axis_spectra(x, 10, 100)
    prob = two_axis_problem(e_r, e_c)
    sol, info = solve_newton(prob)
    assert info.converged and info.n_active > 0
    g, at = _kkt_invariants(prob, sol)
    r1 = len(e_r)
    lhs = g[r1:][at[r1:]].sum() - g[:r1][at[:r1]].sum()
    np.testing.assert_allclose(lhs, e_c.sum() - e_r.sum(), rtol=1e-9)
    # the truncated axis is strictly above its bound; clipping is on mu
    assert not np.any(at[:r1])


def test_rank_one_closed_form():
    # r1 = 1: mu_j(lam) = max(eps, 1/E2_j - lam) and lam solves
    # E1 = sum_j 1/(lam + mu_j(lam)), a monotone 1-D root (bisection).
    rng = np.random.default_rng(10)
    e2 = np.sort(rng.uniform(0.5, 5.0, 40))[::-1]
    e1 = np.array([6.0])
    prob = two_axis_problem(e1, e2)
    eps = prob.eps[1]

    def h(lam):
        mu = np.maximum(eps, 1.0 / e2 - lam)
        return np.sum(1.0 / (lam + mu)) - e1[0]

    lo_, hi_ = prob.eps[0], 1e6
    for _ in range(300):
        mid = 0.5 * (lo_ + hi_)
        if h(mid) > 0:
            lo_ = mid
        else:
            hi_ = mid
    lam = 0.5 * (lo_ + hi_)
    mu = np.maximum(eps, 1.0 / e2 - lam)
    sol, info = solve_newton(prob)
    assert info.converged
    np.testing.assert_allclose(sol[0], lam, rtol=1e-9)
    np.testing.assert_allclose(sol[1:], mu, rtol=1e-8, atol=1e-9 * lam)
    free = mu > eps
    np.testing.assert_allclose(sol[0] + sol[1:][free], 1.0 / e2[free], rtol=1e-9)


def test_scaled_identity_closed_form():
    # X = c I_n, full ranks: S_l = c^2 I, every s_ij = n / c^2; gauge puts
    # min mu at eps.
    n, c = 6, 1.7
    x = c * np.eye(n)
    e_r, _, e_c, _ = two_axis_spectra(x, n, n)
    prob = two_axis_problem(e_r, e_c)
    sol, info = solve_newton(prob)
    s = sol[:n, None] + sol[None, n:]
    np.testing.assert_allclose(s, n / c**2, rtol=1e-10)
    np.testing.assert_allclose(sol[n:].min(), prob.eps[1], rtol=0, atol=1e-15 * s.max())


def test_equal_spectra_give_symmetric_solution():
    # E1 = E2 with full ranks: lam = mu + const (the problem is symmetric).
    x, _, _ = planted_c1()
    e_r, _, e_c, _ = two_axis_spectra(x, 100, 100)
    prob = two_axis_problem(e_r, e_c)
    sol, info = solve_newton(prob)
    assert info.converged
    d = sol[:100] - sol[100:]
    np.testing.assert_allclose(d, d[0], atol=1e-9 * np.abs(sol).max())
    # plain (unprojected) gradient vanishes: no bound is active
    g = gradient(sol, prob)
    assert np.max(np.abs(g) / prob.e_all()) <= 1e-10


def test_mean_value_and_upper_bounds():
    # E1_i = sum_j 1/s_ij  =>  min_j s_ij <= r2/E1_i <= max_j s_ij, and
    # lam_i <= r2 / E1_i (existence lemma) for free i.
    x, _, _ = planted_c1()
    e_r, _, e_c, _ = two_axis_spectra(x, 20, 100)
    prob = two_axis_problem(e_r, e_c)
    sol, info = solve_newton(prob)
    lam, mu = sol[:20], sol[20:]
    s = lam[:, None] + mu[None, :]
    m = 100 / e_r
    assert np.all(s.min(axis=1) <= m * (1 + 1e-9))
    assert np.all(s.max(axis=1) >= m * (1 - 1e-9))
    assert np.all(lam <= m * (1 + 1e-9))


def test_lbfgsb_second_path_agrees():
    x, _, _ = planted_c1()
    e_r, _, e_c, _ = two_axis_spectra(x, 30, 100)
    prob = two_axis_problem(e_r, e_c)
    sol, info = solve_newton(prob)
    lo = prob.lower()
    res = scipy.optimize.minimize(lambda z: objective(z, prob), 1 / prob.e_all(),
                                  jac=lambda z: gradient(z, prob), method="L-BFGS-B",
                                  bounds=list(zip(lo, [None] * prob.n)),
                                  options={"ftol": 1e-16, "gtol": 1e-13, "maxiter": 100000,
                                           "maxcor": 50})
    s1 = sol[:30, None] + sol[None, 30:]
    s2 = res.x[:30, None] + res.x[None, 30:]
    np.testing.assert_allclose(s1, s2, rtol=5e-4)
    assert objective(sol, prob) <= res.fun + 1e-10 * abs(res.fun)


def test_paper_algorithm1_reaches_same_sums():
    rng = np.random.default_rng(11)
    x = rng.standard_normal((12, 8))
    e_r, _, e_c, _ = two_axis_spectra(x, 8, 8)
    prob = two_axis_problem(e_r, e_c)
    sol, _ = solve_newton(prob)
    gd, iters = solve_alg1(prob, tol=1e-9)
    s1 = sol[:8, None] + sol[None, 8:]
    s2 = gd[:8, None] + gd[None, 8:]
    np.testing.assert_allclose(s1, s2, rtol=1e-6)


def test_eps_continuity():
    # eps -> 10 eps moves the sums by O(eps) when bounds are active.
    x, _, _ = planted_c1()
    e_r, _, e_c, _ = two_axis_spectra(x, 10, 100)
    p1 = two_axis_problem(e_r, e_c)
    p2 = two_axis_problem(e_r, e_c, eps=[10 * p1.eps[0]] * 2)
    s1, _ = solve_newton(p1)
    s2, _ = solve_newton(p2)
    a = s1[:10, None] + s1[None, 10:]
    b = s2[:10, None] + s2[None, 10:]
    assert np.max(np.abs(a - b) / a) <= 1e-6


def test_three_axis_full_rank_zero_gradient():
    # A 3-axis tensor at full ranks: all traces equal -> interior optimum,
    # plain gradient zero (the "zero gradient at the optimum" pin).
    from oracle.gram import gram
    rng = np.random.default_rng(12)
    t = rng.standard_normal((4, 5, 6))
    es = [top_eigh(gram(t, a), t.shape[a])[0] for a in range(3)]
    prob = KSProblem(es, [(0, 1, 2)])
    sol, info = solve_newton(prob)
    assert info.converged and info.n_active <= 2
    g = gradient(sol, prob)
    assert np.max(np.abs(g) / prob.e_all()) <= 1e-10
