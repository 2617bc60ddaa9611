"""Pins for the FP64 oracle against facts fixed outside the oracle itself.

Each test checks the oracle against something other than its own formula:
hand-derived cases (tests/golden), library routines (np.cov, eigvalsh, svd),
exhaustive enumeration over the faces of F, the projection's variational
inequality over all vertices of F, finite differences, and the FISTA
Lyapunov inequality.  All run on the CPU in a few seconds.
"""
import json
import os

import numpy as np
import pytest

from synth import CFG_SMALL, countsketch_hash, factor_returns, gaussian_sketch, power_start
from oracle.center import center_factor
from oracle.projection import (PROJ_BRACKET, PROJ_INFEASIBLE, PROJ_OK, active_set, project_F,
                               project_F_dykstra, project_F_safeguarded, project_halfspace,
                               project_simplex)
from oracle.npga import (_lanczos_top, fw_gap, gradient, gradient_sigma, initial_point, kkt_residual,
                         kkt_residual_sigma, lanczos_norm2, lanczos_norm2_sigma, lin_min_F, npga, npga_sigma,
                         objective, objective_sigma, power_norm2, power_norm2_sigma, sigma_from_factor,
                         solver_gap, step_size, vertices_F)
from oracle.bruteforce import project_bruteforce, qp_bruteforce
from oracle import strmodel

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")))


def small_problem(n=30, T=200, seed=3, pct=60.0):
    R = factor_returns(CFG_SMALL.scaled(n, T, seed=seed), np.float32).astype(np.float64)
    mu, L, tr = center_factor(R)
    return R, mu, L, float(np.percentile(mu, pct))


# ---------------------------------------------------------------- centering
def test_center_matches_numpy_cov():
    R, mu, L, _ = small_problem(40, 300)
    np.testing.assert_allclose(L @ L.T, np.cov(R, ddof=1), rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(mu, np.mean(R, axis=1), rtol=1e-13)
    assert np.max(np.abs(L.sum(axis=1))) < 1e-14
    _, _, tr = center_factor(R)
    assert tr == pytest.approx(np.trace(np.cov(R, ddof=1)), rel=1e-12)


def test_objective_matches_explicit_sigma():
    R, mu, L, _ = small_problem(CFG_SMALL.n, CFG_SMALL.T)
    Sigma = np.cov(R, ddof=1)
    x = np.random.default_rng(0).dirichlet(np.ones(L.shape[0]))
    assert objective(L, 0.0, x) == pytest.approx(x @ Sigma @ x, rel=1e-12)
    assert objective(L, 0.3, x) == pytest.approx(x @ Sigma @ x + 0.3 * x @ x, rel=1e-12)


@pytest.mark.parametrize("gamma", [0.0, 2e-4])
def test_gradient_matches_finite_differences(gamma):
    _, _, L, _ = small_problem(12, 80)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(12)
    g = gradient(L, gamma, x)
    h = 1e-6
    fd = np.array([(objective(L, gamma, x + h * e) - objective(L, gamma, x - h * e)) / (2 * h)
                   for e in np.eye(12)])
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-12)


# --------------------------------------------------------------- projection
@pytest.mark.parametrize("case", GOLD["simplex"])
def test_simplex_hand_cases(case):
    x, tau = project_simplex(np.array(case["v"]))
    np.testing.assert_allclose(x, case["x"], atol=1e-15)
    assert tau == pytest.approx(case["tau"], abs=1e-15)


@pytest.mark.parametrize("case", GOLD["projection_F"])
def test_projection_hand_cases(case):
    p = project_F(np.array(case["v"]), np.array(case["mu"]), case["R"], case["mode"])
    assert p.status == PROJ_OK
    np.testing.assert_allclose(p.x, case["x"], atol=1e-13)
    if case["nu"] is not None:
        assert p.nu == pytest.approx(case["nu"], rel=1e-10, abs=1e-12)
        assert p.tau == pytest.approx(case["tau"], rel=1e-10, abs=1e-12)


def test_simplex_matches_bruteforce_and_fixes_simplex_points():
    rng = np.random.default_rng(2)
    for n in range(1, 8):
        for _ in range(20):
            v = rng.standard_normal(n)
            x, _ = project_simplex(v)
            # R below min mu: F is the whole simplex.
            ref = project_bruteforce(v, np.zeros(n), -1.0)
            np.testing.assert_allclose(x, ref, atol=1e-12)
        p = rng.dirichlet(np.ones(n))
        np.testing.assert_allclose(project_simplex(p)[0], p, atol=1e-15)


def test_halfspace_closed_form():
    rng = np.random.default_rng(3)
    mu = rng.uniform(0.0, 0.01, 9)
    y = rng.standard_normal(9)
    R = float(mu @ y) + 0.05
    p = project_halfspace(y, mu, R)
    assert mu @ p == pytest.approx(R, rel=1e-13)
    d = p - y                      # the move is along mu
    np.testing.assert_allclose(d / np.linalg.norm(d), mu / np.linalg.norm(mu), atol=1e-12)
    np.testing.assert_allclose(project_halfspace(p, mu, R), p, atol=0)


@pytest.mark.parametrize("mode", ["ge", "eq"])
def test_projection_matches_bruteforce(mode):
    rng = np.random.default_rng(4 if mode == "ge" else 5)
    checked = 0
    for _ in range(150):
        n = int(rng.integers(1, 8))
        v = rng.standard_normal(n) * 0.5
        mu = rng.uniform(-1e-3, 2e-3, n)
        R = float(rng.uniform(mu.min(), mu.max())) if n > 1 else float(mu[0])
        p = project_F(v, mu, R, mode)
        ref = project_bruteforce(v, mu, R, mode)
        assert p.status == PROJ_OK
        np.testing.assert_allclose(p.x, ref, atol=1e-10)
        checked += 1
    assert checked == 150


def test_projection_variational_inequality_over_all_vertices():
    rng = np.random.default_rng(6)
    for n in (50, 200, 400):
        mu = rng.uniform(-2e-4, 6e-4, n)
        v = rng.standard_normal(n) * 3e-3 + 1.0 / n
        R = float(np.percentile(mu, 80))
        p = project_F(v, mu, R)
        assert p.status == PROJ_OK
        x = p.x
        assert x.min() >= 0 and abs(x.sum() - 1) < 1e-13 and mu @ x >= R - 1e-15
        # <v - p, q - p> <= 0 for every vertex q of F (exact for a polytope).
        r = v - x
        worst = -np.inf
        for i, j, lam in vertices_F(mu, R):
            q = np.zeros(n)
            q[i] += lam
            q[j] += 1.0 - lam
            worst = max(worst, float(r @ (q - x)))
        assert worst <= 1e-14


def test_phi_is_nondecreasing_in_nu():
    rng = np.random.default_rng(7)
    mu = rng.uniform(-2e-4, 6e-4, 300)
    v = rng.standard_normal(300) * 1e-3
    nus = np.linspace(0.0, 50.0, 400)
    phi = [float(mu @ project_simplex(v + nu * mu)[0]) for nu in nus]
    assert np.all(np.diff(phi) >= -1e-18)


def test_projection_edge_cases():
    mu = np.array([0.01, 0.02, 0.03])
    v = np.array([0.2, 0.3, 0.5])
    assert project_F(v, mu, 0.031).status == PROJ_INFEASIBLE
    assert project_F(v, mu, 0.005, "eq").status == PROJ_INFEASIBLE
    # Equality mode with a target below mu^T Pi_Delta(v): nu < 0.
    p = project_F(v, mu, 0.015, "eq")
    assert p.status == PROJ_OK and p.nu < 0 and mu @ p.x == pytest.approx(0.015, abs=1e-15)
    np.testing.assert_allclose(p.x, project_bruteforce(v, mu, 0.015, "eq"), atol=1e-12)
    # n = 1: the only feasible point.
    p = project_F(np.array([-3.0]), np.array([1e-3]), 5e-4)
    assert p.status == PROJ_OK and p.x[0] == 1.0
    # Ties in v and mu are harmless: the projection is unique.
    vv = np.array([0.3, 0.3, 0.3, 0.1])
    mm = np.array([0.01, 0.01, 0.02, 0.02])
    p = project_F(vv, mm, 0.018)
    np.testing.assert_allclose(p.x, project_bruteforce(vv, mm, 0.018), atol=1e-12)
    act, deg = active_set(vv, mm, p.nu, p.tau)
    assert np.array_equal(act[~deg], (p.x > 0)[~deg])


# --------------------------------------------------------- power and NPGA
def test_power_method_approaches_lambda_max_from_below():
    _, _, L, _ = small_problem(CFG_SMALL.n, CFG_SMALL.T)
    lam_max = np.linalg.eigvalsh(L @ L.T)[-1]
    r = power_start(L.shape[0])
    prev = 0.0
    for it in (1, 2, 5, 10, 50, 200, 1500):
        lam = power_norm2(L, r, it)
        assert lam <= lam_max * (1 + 1e-12)
        assert lam >= prev * (1 - 1e-12)        # Rayleigh quotient increases
        prev = lam
    # The top eigenvalues of this panel are clustered, so convergence is slow.
    assert prev == pytest.approx(lam_max, rel=1e-9)
    assert step_size(lam_max, 0.0, 0.0) == pytest.approx(1.0 / (2.0 * lam_max))


def test_lanczos_exact_after_n_steps():
    # In exact arithmetic n Lanczos steps span R^n, so the tridiagonal matrix
    # is similar to A and its top eigenvalue is lambda_max; a dropped
    # beta q_{j-1} term or a wrong alpha_j breaks that.
    rng = np.random.default_rng(5)
    for n in (1, 2, 6, 9):
        L = rng.standard_normal((n, 3 * n + 1))
        lam_max = np.linalg.eigvalsh(L @ L.T)[-1]
        r = rng.standard_normal(n)
        assert lanczos_norm2(L, r, n) == pytest.approx(lam_max, rel=1e-10)
        # more steps than n: the recurrence stops at the invariant space
        assert lanczos_norm2(L, r, n + 5) == pytest.approx(lam_max, rel=1e-10)


def test_lanczos_breakdown_on_invariant_krylov_space():
    # A = diag(9, 4, 0, 0, 0): from r = 1 the Krylov space has dimension 3
    # (one direction per distinct eigenvalue), so beta_4 = 0 and the estimate
    # is exactly 9 after three steps.
    L = np.zeros((5, 2))
    L[0, 0], L[1, 1] = 3.0, 2.0
    top, k = _lanczos_top(lambda q: L @ (L.T @ q), np.ones(5), 25)
    assert k == 3
    assert top == pytest.approx(9.0, rel=1e-14)
    assert lanczos_norm2(L, np.zeros(5), 10) == 0.0        # zero start: no direction


def test_lanczos_bounds_power_method_and_lambda_max():
    # The k-step value maximises the Rayleigh quotient over K_k(A, r), which
    # holds the power iterate after k - 1 steps, and lies below lambda_max.
    _, _, L, _ = small_problem(CFG_SMALL.n, CFG_SMALL.T)
    lam_max = np.linalg.eigvalsh(L @ L.T)[-1]
    r = power_start(L.shape[0])
    prev = 0.0
    for k in (1, 2, 3, 5, 8, 12, 20, 30):
        lz = lanczos_norm2(L, r, k)
        assert lz >= power_norm2(L, r, k - 1) * (1 - 1e-12)
        assert lz <= lam_max * (1 + 1e-12)
        assert lz >= prev * (1 - 1e-12)
        prev = lz
    # far fewer products than the power method for the same accuracy on
    # this clustered spectrum
    assert lanczos_norm2(L, r, 30) >= power_norm2(L, r, 200) * (1 - 1e-12)
    S = sigma_from_factor(L)
    assert lanczos_norm2_sigma(S, r, 12) == pytest.approx(lanczos_norm2(L, r, 12), rel=1e-10)


def test_npga_hand_case():
    c = GOLD["npga"][0]
    L, mu = np.array(c["L"]), np.array(c["mu"])
    lam = power_norm2(L, np.array([1.0, 1.0]), 50)
    x0 = initial_point(mu, c["R"])
    res = npga(L, 0.0, mu, c["R"], x0, step_size(lam, 0.0), eps=1e-12, max_iter=5000)
    assert res.converged
    np.testing.assert_allclose(res.x, c["x"], atol=1e-10)
    assert res.f == pytest.approx(c["f"], rel=1e-9)


@pytest.mark.parametrize("gamma", [0.0, 5e-5])
def test_npga_matches_bruteforce_qp(gamma):
    for seed in range(4):
        n = 6 + seed % 3
        R, mu, L, Rt = small_problem(n, 60, seed=10 + seed, pct=70)
        Sigma = L @ L.T + gamma * np.eye(n)
        ref = qp_bruteforce(Sigma, mu, Rt)
        lam = power_norm2(L, power_start(n), 200)
        x0 = initial_point(mu, Rt)
        res = npga(L, gamma, mu, Rt, x0, step_size(lam, gamma), eps=1e-11, max_iter=200000)
        assert res.converged
        np.testing.assert_allclose(res.x, ref, atol=1e-7)
        gap = fw_gap(L, gamma, mu, Rt, res.x)
        f_star = float(ref @ Sigma @ ref)
        assert -1e-18 <= res.f - f_star <= gap + 1e-18


def test_npga_fista_lyapunov_inequality():
    """Beck--Teboulle (2009) Lemma 4.1 holds along Algorithm 1's iterates.

    With v_k = f(x^k) - f*, u_k = t_{k-1} x^k - (t_{k-1} - 1) x^{k-1} - x*:
    2 alpha t_{k-1}^2 v_k + ||u_k||^2 is nonincreasing for alpha <= 1/L_f.
    A wrong momentum, step or extrapolation breaks it on these
    ill-conditioned 8-asset, 10-period panels (condition numbers 1e2..2e3).
    """
    for seed in (20, 22, 23, 24, 25):
        R, mu, L, Rt = small_problem(8, 10, seed=seed, pct=65)
        Sigma = L @ L.T
        xs = qp_bruteforce(Sigma, mu, Rt)
        fs = float(xs @ Sigma @ xs)
        alpha = 1.0 / (2.0 * np.linalg.eigvalsh(Sigma)[-1])
        x0 = initial_point(mu, Rt)
        K = 150
        traj = npga(L, 0.0, mu, Rt, x0, alpha, eps=0.0, max_iter=K, kkt_every=0,
                    record=True).trajectory
        assert len(traj) == K + 1 and np.array_equal(traj[0], x0)
        t = [1.0]
        for _ in range(K + 1):
            t.append(0.5 * (1 + np.sqrt(1 + 4 * t[-1] ** 2)))
        E = []
        for k in range(1, K + 1):
            u = t[k - 1] * traj[k] - (t[k - 1] - 1) * traj[k - 1] - xs
            E.append(2 * alpha * t[k - 1] ** 2 * (objective(L, 0.0, traj[k]) - fs) + u @ u)
        assert np.max(np.diff(E)) <= 1e-9 * max(E)
        # And the O(1/k^2) rate of Theorem 1(a): f - f* <= 2||x^0 - x*||^2 / (alpha (k+1)^2).
        for k in range(1, K + 1):
            assert objective(L, 0.0, traj[k]) - fs <= 2 * (x0 - xs) @ (x0 - xs) / (alpha * (k + 1) ** 2)


def test_npga_linear_rate_with_ridge():
    """With gamma > 0 the KKT residual decays geometrically (Theorem 1(b) regime)."""
    R, mu, L, Rt = small_problem(60, 300, seed=5)
    gamma = 5e-4
    lam = power_norm2(L, power_start(60), 100)
    x0 = initial_point(mu, Rt)
    res = npga(L, gamma, mu, Rt, x0, step_size(lam, gamma), eps=1e-13, max_iter=3000, kkt_every=1)
    assert res.converged
    ks = np.array([k for k, _ in res.kkt_history[5:]])
    rs = np.array([r for _, r in res.kkt_history[5:]])
    slope = np.polyfit(ks, np.log(np.maximum(rs, 1e-300)), 1)[0]
    assert slope < -0.02


def test_npga_small_config_kkt_and_certificates():
    R, mu, L, Rt = small_problem(CFG_SMALL.n, CFG_SMALL.T, seed=CFG_SMALL.seed)
    lam = power_norm2(L, power_start(L.shape[0]), 50)
    a = step_size(lam, 0.0)
    x0 = initial_point(mu, Rt)
    res = npga(L, 0.0, mu, Rt, x0, a, eps=1e-6, max_iter=20000)
    assert res.converged and res.kkt <= 1e-6
    x = res.x
    assert x.min() >= 0 and abs(x.sum() - 1) < 1e-12 and mu @ x >= Rt - 1e-15
    assert kkt_residual(L, 0.0, mu, Rt, x, a) == pytest.approx(res.kkt)
    # FW gap bounds f - f*; a long run gives f* from below within it.
    gap = fw_gap(L, 0.0, mu, Rt, x)
    ref = npga(L, 0.0, mu, Rt, x0, a, eps=1e-12, max_iter=200000)
    assert 0.0 <= res.f - ref.f <= gap + 1e-18
    assert solver_gap(res.f, ref.f) < 1e-3


def test_lin_min_F_matches_vertex_scan_and_gap_metric():
    rng = np.random.default_rng(9)
    mu = rng.uniform(-1e-3, 1e-3, 40)
    g = rng.standard_normal(40)
    R = 2e-4
    best = min(lam * g[i] + (1 - lam) * g[j] for i, j, lam in vertices_F(mu, R))
    assert lin_min_F(g, mu, R) == pytest.approx(best, abs=1e-15)
    assert solver_gap(1.1, 1.0) == pytest.approx(0.1)
    assert solver_gap(0.9, 1.0) == 0.0
    assert solver_gap(1.0, 0.0) == pytest.approx(1e12)


# ------------------------------------------------- explicit Sigma (Sec. 3)
def test_sigma_form_matches_covariance_and_bruteforce():
    """Sigma = L L^T is np.cov; its objective, gradient (FD) and power estimate
    agree with the library; NPGA on Sigma reaches the exhaustive QP optimum."""
    R, mu, L, Rt = small_problem(40, 300, seed=4)
    S = sigma_from_factor(L)
    np.testing.assert_allclose(S, np.cov(R, ddof=1), rtol=1e-12, atol=1e-18)
    x = np.random.default_rng(3).dirichlet(np.ones(40))
    assert objective_sigma(S, 0.2, x) == pytest.approx(x @ np.cov(R, ddof=1) @ x + 0.2 * x @ x, rel=1e-12)
    h = 1e-6
    fd = np.array([(objective_sigma(S, 0.2, x + h * e) - objective_sigma(S, 0.2, x - h * e)) / (2 * h)
                   for e in np.eye(40)])
    np.testing.assert_allclose(gradient_sigma(S, 0.2, x), fd, rtol=1e-6, atol=1e-12)
    lam_max = np.linalg.eigvalsh(S)[-1]
    prev = 0.0
    for it in (1, 5, 50, 2000):
        lam = power_norm2_sigma(S, power_start(40), it)
        assert prev * (1 - 1e-12) <= lam <= lam_max * (1 + 1e-12)
        prev = lam
    assert prev == pytest.approx(lam_max, rel=1e-9)
    for gamma in (0.0, 5e-5):
        for seed in range(3):
            n = 6 + seed
            _, mu, L, Rt = small_problem(n, 60, seed=30 + seed, pct=70)
            S = sigma_from_factor(L)
            ref = qp_bruteforce(S + gamma * np.eye(n), mu, Rt)
            a = step_size(np.linalg.eigvalsh(S)[-1], gamma)
            res = npga_sigma(S, gamma, mu, Rt, initial_point(mu, Rt), a, eps=1e-11, max_iter=200000)
            assert res.converged
            np.testing.assert_allclose(res.x, ref, atol=1e-7)
            assert kkt_residual_sigma(S, gamma, mu, Rt, res.x, a) == pytest.approx(res.kkt)


# -------------------------------------------- step and momentum variants (Sec. 3.1)
def test_constant_momentum_linear_rate():
    """The strongly convex specialisation (beta = (1 - q)/(1 + q), q = sqrt(alpha m_f))
    obeys the V-FISTA bound f(x^k) - f* <= (1 - q)^k (f(x^0) - f* + m_f/2 ||x^0 - x*||^2)
    (Beck, First-Order Methods in Optimization, Thm. 10.7.7) with m_f = 2 (lambda_min + gamma);
    a wrong beta or a missing extrapolation breaks it."""
    for seed, gamma in ((40, 2e-5), (41, 1e-4), (42, 5e-6)):
        _, mu, L, Rt = small_problem(8, 40, seed=seed, pct=65)
        S = sigma_from_factor(L)
        ev = np.linalg.eigvalsh(S)
        Lf, mf = 2 * (ev[-1] + gamma), 2 * (ev[0] + gamma)
        a = 1.0 / Lf
        xs = qp_bruteforce(S + gamma * np.eye(8), mu, Rt)
        fs = objective_sigma(S, gamma, xs)
        x0 = initial_point(mu, Rt)
        K = 400
        traj = npga(L, gamma, mu, Rt, x0, a, eps=0.0, max_iter=K, kkt_every=0, record=True,
                    momentum="constant", m_f=mf).trajectory
        q = np.sqrt(a * mf)
        c0 = objective_sigma(S, gamma, x0) - fs + 0.5 * mf * (x0 - xs) @ (x0 - xs)
        for k in range(1, K + 1):
            assert objective_sigma(S, gamma, traj[k]) - fs <= (1 - q) ** k * c0 + 1e-17
        # the Sigma form follows the same iterates
        traj2 = npga_sigma(S, gamma, mu, Rt, x0, a, eps=0.0, max_iter=K, kkt_every=0, record=True,
                           momentum="constant", m_f=mf).trajectory
        assert max(np.max(np.abs(u - w)) for u, w in zip(traj, traj2)) <= 1e-12


def test_backtracking_rule():
    """A trial step at or below 1/L_f is never shrunk (the iterates are the fixed-step ones);
    from a 100x too long trial the accepted step stays in [rho/L_f, 100/L_f], every accepted
    step satisfies the sufficient-decrease inequality, and the run reaches the exhaustive optimum."""
    _, mu, L, Rt = small_problem(8, 50, seed=44, pct=70)
    S = sigma_from_factor(L)
    Lf = 2 * np.linalg.eigvalsh(S)[-1]
    x0 = initial_point(mu, Rt)
    fixed = npga(L, 0.0, mu, Rt, x0, 1.0 / Lf, eps=0.0, max_iter=60, kkt_every=0, record=True)
    bt = npga(L, 0.0, mu, Rt, x0, 0.0, eps=0.0, max_iter=60, kkt_every=0, record=True,
              backtrack=(1.0 / Lf, 0.5))
    assert bt.alpha == 1.0 / Lf
    assert all(np.array_equal(u, w) for u, w in zip(fixed.trajectory, bt.trajectory))
    rho = 0.6
    res = npga(L, 0.0, mu, Rt, x0, 0.0, eps=1e-11, max_iter=200000, backtrack=(100.0 / Lf, rho))
    assert rho / Lf <= res.alpha <= 100.0 / Lf and res.alpha < 100.0 / Lf
    assert res.converged
    np.testing.assert_allclose(res.x, qp_bruteforce(S, mu, Rt), atol=1e-7)
    # the printed inequality holds on an accepted step, and the evaluated quadratic form equals it
    d = np.random.default_rng(2).standard_normal(8)
    y = np.random.default_rng(3).standard_normal(8)
    lhs = objective_sigma(S, 3e-5, y + d) - objective_sigma(S, 3e-5, y) - gradient_sigma(S, 3e-5, y) @ d
    assert lhs == pytest.approx(objective(L, 3e-5, d), rel=1e-9)
    short = npga_sigma(S, 0.0, mu, Rt, x0, 0.0, eps=0.0, max_iter=1, kkt_every=0, record=True,
                       backtrack=(100.0 / Lf, rho))
    y, x1, a1 = x0, short.trajectory[1], short.alpha
    d = x1 - y
    assert objective_sigma(S, 0.0, x1) <= (objective_sigma(S, 0.0, y) + gradient_sigma(S, 0.0, y) @ d
                                           + d @ d / (2 * a1)) * (1 + 1e-12)
    # the step before the accepted one failed the test (or was the first trial)
    if a1 < 100.0 / Lf:
        a0 = a1 / rho
        p0 = project_F(y - a0 * gradient_sigma(S, 0.0, y), mu, Rt).x
        d0 = p0 - y
        assert objective_sigma(S, 0.0, p0) > (objective_sigma(S, 0.0, y) + gradient_sigma(S, 0.0, y) @ d0
                                              + d0 @ d0 / (2 * a0))


@pytest.mark.parametrize("mode", ["ge", "eq"])
def test_dykstra_safeguard_matches_exact_projection(mode):
    """Dykstra's alternating projections reach the exhaustive-search projection;
    with a one-step bracketing budget the safeguarded projector falls back to it.
    mu is drawn with both signs, so H is not nearly parallel to the simplex
    plane (where alternating projections crawl)."""
    rng = np.random.default_rng(17)
    fell_back = 0
    for _ in range(20):
        n = int(rng.integers(2, 9))
        v = rng.standard_normal(n) * 0.4
        mu = np.sort(rng.uniform(-1.0, 1.0, n)) * 1e-2
        mu[0], mu[-1] = -abs(mu[0]) - 2e-3, abs(mu[-1]) + 2e-3
        R = float(np.quantile(mu, rng.uniform(0.3, 0.95)))
        ref = project_bruteforce(v, mu, R, mode)
        xd, sweeps = project_F_dykstra(v, mu, R, mode)
        assert sweeps < 100000
        np.testing.assert_allclose(xd, ref, atol=1e-9)
        b = project_F(v, mu, R, mode, max_bracket=1)
        r = project_F_safeguarded(v, mu, R, mode, max_bracket=1)
        fell_back += b.status == PROJ_BRACKET
        assert r.status == PROJ_OK
        np.testing.assert_allclose(r.x, ref, atol=1e-9)
    assert fell_back >= 5


# ---------------------------------------------------------------- STR
def test_str_spectrum_identities():
    _, _, L, _ = small_problem(60, 400, seed=2)
    Phi_t = gaussian_sketch(400, 120, seed=3)
    Lt = strmodel.sketch(L, Phi_t)
    k = 10
    L_eff, sigma, Uk = strmodel.truncate(Lt, k)
    # Library SVD of tilde L gives the same singular values.
    sv = np.linalg.svd(Lt, compute_uv=False)
    np.testing.assert_allclose(sigma, sv[:k], rtol=1e-10)
    np.testing.assert_allclose(L_eff.T @ L_eff, np.diag(sigma ** 2), atol=1e-12 * sigma[0] ** 2)
    gamma = strmodel.ridge_default(np.sum(L * L), 60)
    Sh = strmodel.str_covariance(L_eff, gamma)
    ev = np.sort(np.linalg.eigvalsh(Sh))[::-1]
    want = np.sort(np.concatenate([sigma ** 2 + gamma, np.full(60 - k, gamma)]))[::-1]
    np.testing.assert_allclose(ev, want, rtol=1e-9, atol=1e-12 * ev[0])
    assert ev[0] / ev[-1] == pytest.approx((sigma[0] ** 2 + gamma) / gamma, rel=1e-8)
    # hat L hat L^T = hat Sigma with V_l from the SVD of tilde L (App. D.3).
    _, _, Vt = np.linalg.svd(Lt, full_matrices=False)
    Lhat = strmodel.structured_factor(L, Phi_t, Vt[:k].T, gamma)
    np.testing.assert_allclose(Lhat @ Lhat.T, Sh, rtol=1e-9, atol=1e-12 * ev[0])
    # Truncation error is lambda_{l+1} of tilde Sigma (Eckart--Young).
    Kt = Lt @ Lt.T
    assert np.linalg.norm(Kt - L_eff @ L_eff.T, 2) == pytest.approx(sv[k] ** 2, rel=1e-8)


def test_sketch_embedding_bound_and_moments():
    rng_shape = (80, 3000)
    _, _, L, _ = small_problem(*rng_shape, seed=4)
    s = 1500
    Phi_t = gaussian_sketch(rng_shape[1], s, seed=5)
    # Moments of Phi: mean 0, variance 1/s.
    assert abs(Phi_t.mean()) < 5.0 / np.sqrt(Phi_t.size) / np.sqrt(s)
    assert Phi_t.var() * s == pytest.approx(1.0, rel=0.01)
    Sigma = L @ L.T
    Lt = strmodel.sketch(L, Phi_t)
    # Empirical epsilon of the subspace embedding for Im(L^T).
    U, _, _ = np.linalg.svd(L.T, full_matrices=False)
    G = (Phi_t @ U)
    eps = np.linalg.norm(G.T @ G - np.eye(U.shape[1]), 2)
    assert eps < 1.0
    assert np.linalg.norm(Lt @ Lt.T - Sigma, 2) <= eps * np.linalg.norm(Sigma, 2) * (1 + 1e-10)
    x = np.random.default_rng(1).dirichlet(np.ones(80))
    q, qt = x @ Sigma @ x, np.sum((Lt.T @ x) ** 2)
    assert (1 - eps) * q <= qt <= (1 + eps) * q


def test_countsketch_map_and_embedding():
    """CountSketch (Sec. 2.3 (2)): one signed nonzero per row of Phi; an
    injective hash makes Phi a signed partial permutation, so the sketch keeps
    the covariance exactly; over independent draws tilde L tilde L^T is
    unbiased for L L^T (E[Phi Phi^T] = I); per column, tilde L is the signed
    bucket sum checked element by element on a hand case."""
    h, sg = countsketch_hash(5000, 64, seed=4)
    assert h.min() >= 0 and h.max() < 64 and set(np.unique(sg)) == {-1, 1}
    assert abs(np.mean(sg)) < 0.05 and np.all(np.bincount(h, minlength=64) > 0)
    Phi = strmodel.countsketch_matrix(h, sg, 64)
    assert np.array_equal((Phi != 0).sum(axis=1), np.ones(5000))
    # hand case: T = 5, s = 3
    L = np.array([[1.0, 2.0, 3.0, 4.0, 5.0], [0.5, -1.0, 0.0, 2.0, 1.0]])
    hh, ss = np.array([2, 0, 2, 1, 0]), np.array([1, -1, -1, 1, 1])
    np.testing.assert_array_equal(strmodel.countsketch(L, hh, ss, 3),
                                  [[-2.0 + 5.0, 4.0, 1.0 - 3.0], [1.0 + 1.0, 2.0, 0.5]])
    # injective hash: exact covariance
    _, _, L, _ = small_problem(20, 80, seed=6)
    perm = np.random.default_rng(1).permutation(100)[:80]
    sgn = np.where(np.random.default_rng(2).random(80) < 0.5, -1, 1)
    Lt = strmodel.countsketch(L, perm, sgn, 100)
    np.testing.assert_allclose(Lt @ Lt.T, L @ L.T, rtol=1e-12, atol=1e-20)
    # unbiased over draws (Monte Carlo, 400 draws, s = 40 < T = 80)
    acc = np.zeros((20, 20))
    for d in range(400):
        hh, ss = countsketch_hash(80, 40, seed=100 + d)
        Lt = strmodel.countsketch(L, hh, ss, 40)
        acc += Lt @ Lt.T
    acc /= 400
    S = L @ L.T
    assert np.max(np.abs(acc - S)) <= 0.02 * np.max(np.abs(S))      # dropping the signs gives 0.035


def test_knee_rank_and_kappa_ridge():
    lam = np.array([100.0, 50.0, 40.0, 5.0, 4.9, 4.8, 0.1])
    # lam_{i+1}/lam_i = .5 .8 .125 .98 .98 .02 and lam_i/lam_1 = 1 .5 .4 .05 .049 .048:
    # with rho = .6, tau = .1 admits i in {1, 3}; tau = 1e-2 also admits i = 6.
    assert strmodel.knee_rank(lam, 0.1, 0.6) == 3
    assert strmodel.knee_rank(lam, 1e-2, 0.6) == 6
    g = strmodel.gamma_for_kappa(10.0, 101.0)
    assert (100.0 + g) / g == pytest.approx(101.0)


def test_product_at_x_by_linearity_along_the_iterates():
    """Sec. 3.1 tests the KKT condition at x^k while Algorithm 1 forms the
    gradient at y^k.  Since y^k = (1 + beta_{k-1}) x^k - beta_{k-1} x^{k-1},
    L L^T x^k = (L L^T y^k + beta_{k-1} L L^T x^{k-1}) / (1 + beta_{k-1}) with
    L L^T x^0 = L L^T y^0; the objective x^T (L L^T x) + gamma ||x||^2 follows
    from the same product.  Checked along a recorded FISTA run against the
    direct products (a beta off by one iteration fails it)."""
    rng = np.random.default_rng(11)
    n, T, gamma = 30, 80, 1e-3
    L = rng.standard_normal((n, T)) * 0.1
    mu = rng.uniform(-2e-4, 6e-4, n)
    R = float(np.percentile(mu, 60))
    a = step_size(power_norm2(L, rng.standard_normal(n), 50), gamma)
    res = npga(L, gamma, mu, R, initial_point(mu, R), a, eps=0.0, max_iter=40, record=True)
    X = res.trajectory
    assert len(X) == 41
    t, beta_prev, gx = 1.0, 0.0, None
    for k, xk in enumerate(X):
        y = xk if k == 0 else xk + beta_prev * (xk - X[k - 1])
        gy = L @ (L.T @ y)
        gx = gy if k == 0 else (gy + beta_prev * gx) / (1.0 + beta_prev)
        direct = L @ (L.T @ xk)
        assert np.max(np.abs(gx - direct)) <= 1e-12 * np.max(np.abs(direct))
        assert xk @ gx + gamma * (xk @ xk) == pytest.approx(objective(L, gamma, xk), rel=1e-12)
        t_new = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        beta_prev, t = (t - 1.0) / t_new, t_new
    assert beta_prev > 0.5                      # momentum well away from 0 by the end


# ------------------------------------------------------------------ counter-based draws (oracle/rng.py)
def test_philox_known_answers():
    """Philox4x32-10 known-answer vectors published with the generator
    (Salmon et al., SC'11; the Random123 known-answer tests): zero counter
    and key, all-ones counter and key, and the pi-digit counter and key."""
    from oracle.rng import philox4x32_10
    cases = [((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
             ((0xFFFFFFFF,) * 4, (0xFFFFFFFF, 0xFFFFFFFF), (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
             ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
              (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1))]
    for ctr, key, want in cases:
        got = tuple(int(w) for w in philox4x32_10(*ctr, key))
        assert got == want


def test_gaussian_sketch_draw_is_a_jl_gaussian():
    """Entries of Phi are i.i.d. N(0, 1/s) (Sec. 2.3): mean, variance and the
    normal law (Kolmogorov--Smirnov), E[Phi Phi^T] = I over the s columns, one
    seed gives one matrix (any subset of rows reproduces it) and another
    seed another one."""
    from scipy import stats
    from oracle.rng import gaussian_sketch_t
    s, T = 256, 4003
    P = gaussian_sketch_t(11, s, T)
    assert P.shape == (s, T) and np.all(np.isfinite(P))
    z = P.reshape(-1) * np.sqrt(s)
    N = z.size
    assert abs(z.mean()) < 5.0 / np.sqrt(N)
    assert abs(z.var() - 1.0) < 5.0 * np.sqrt(2.0 / N)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # the four normals of one Philox block are independent: no correlation between t mod 4 lanes
    lanes = z[: (N // 4) * 4].reshape(-1, 4)
    C = np.corrcoef(lanes.T)
    assert np.max(np.abs(C - np.eye(4))) < 5.0 / np.sqrt(lanes.shape[0])
    G = P.T[:64] @ P.T[:64].T                  # rows of Phi (periods): E[Phi Phi^T] = I
    assert np.max(np.abs(np.diag(G) - 1.0)) < 6.0 * np.sqrt(2.0 / s)
    np.testing.assert_array_equal(gaussian_sketch_t(11, s, T, rows=[3, 200]), P[[3, 200]])
    np.testing.assert_array_equal(gaussian_sketch_t(11, s, T), P)
    assert not np.array_equal(gaussian_sketch_t(12, 4, T), P[:4])


def test_countsketch_draw_uniform_buckets_and_signs():
    """h(t) uniform on [0, s), s_t = +-1 with probability 1/2 each, and one
    draw per seed."""
    from scipy import stats
    from oracle.rng import countsketch_draw
    T, s = 200000, 64
    h, sg = countsketch_draw(9, T, s)
    assert h.min() >= 0 and h.max() < s and set(np.unique(sg)) == {-1, 1}
    assert stats.chisquare(np.bincount(h, minlength=s)).pvalue > 1e-3
    assert abs(sg.mean()) < 5.0 / np.sqrt(T)
    h2, sg2 = countsketch_draw(9, T, s)
    assert np.array_equal(h, h2) and np.array_equal(sg, sg2)
    assert not np.array_equal(countsketch_draw(10, T, s)[0], h)


def test_round_bf16_nearest_even():
    """round_bf16 keeps 8 significant bits, rounds to the nearest such value
    and breaks ties to the even one (hand-made ties and random values)."""
    from oracle.rng import round_bf16
    x = np.random.default_rng(5).standard_normal(20000) * 10.0 ** np.random.default_rng(6).integers(-8, 8, 20000)
    r = round_bf16(x)
    m, e = np.frexp(r)
    assert np.all(m * 256.0 == np.rint(m * 256.0))                 # 8 significant bits
    half = np.ldexp(1.0, np.frexp(x)[1] - 9)                        # half a BF16 step at x
    assert np.all(np.abs(r - x) <= half)
    # ties: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 -> even (1); 1 + 3 * 2^-8 -> 1 + 2^-6
    assert round_bf16(1.0 + 2.0 ** -8) == 1.0 and round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert round_bf16(-(1.0 + 2.0 ** -8)) == -1.0 and round_bf16(0.0) == 0.0
