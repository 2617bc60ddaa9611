"""NPGA (Algorithm 1) and its certificates -- test oracle, FP64.

* ``objective`` / ``gradient`` -- Eq. npga-unified-grad:
  f(x) = ||L_eff^T x||^2 + gamma ||x||^2,  grad f(x) = 2 L_eff (L_eff^T x) + 2 gamma x.
* ``power_norm2`` -- the power method of the Sec. 3.1 remark:
  u <- L(L^T u)/||L(L^T u)||, u^0 = r/||r||; returns ||L^T u||^2, an
  estimate of ||L_eff||_2^2.
* ``lanczos_norm2`` -- the other estimate the Sec. 3.1 fixed step names,
  the largest singular value of L_eff, taken as the largest eigenvalue of
  the k x k tridiagonal matrix that k steps of the Lanczos three-term
  recurrence build for A = L L^T from q_1 = r/||r||:
  alpha_j = q_j^T A q_j, r_j = A q_j - alpha_j q_j - beta_j q_{j-1},
  beta_{j+1} = ||r_j||, q_{j+1} = r_j / beta_{j+1}; no reorthogonalisation.
  It stops early when beta_{j+1} vanishes (K_j is invariant under A and the
  estimate is exact).  Its k-step value is the largest Rayleigh quotient over
  the Krylov space K_k(A, r), so it is never below the power method's
  estimate after k - 1 steps (a vector of that space) and never above
  ||L||_2^2.
* ``step_size`` -- fixed step alpha = 1/L_f with L_f = 2(||L_eff||_2^2 + gamma)
  (Sec. 3.1, fixed step).  Reading: the power estimate is raised by a safety
  factor (1 + safety) because the power method approaches ||L||^2 from below.
* ``npga`` -- Algorithm 1 as printed: t_0 = 1, y^0 = x^0; gradient at y^k,
  gradient step, projection onto F, t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2,
  beta_k = (t_k - 1)/t_{k+1}, y^{k+1} = x^{k+1} + beta_k (x^{k+1} - x^k).
  Stops when ||Pi_F(x^k - alpha grad f(x^k)) - x^k||_2 <= eps, checked every
  ``kkt_every`` iterations (Sec. 5.2 uses 5), and returns x^k.
* ``fw_gap`` -- Frank--Wolfe duality gap <g, x> - min_{q in F} <g, q>, an
  upper bound on f(x) - f* for convex f; the linear minimisation is done
  exactly over the vertex list of F.
* ``solver_gap`` -- the relative gap metric of Sec. 5.2.

Explicit covariance (the Sec. 3 remark that NPGA applies unchanged to the
classical model with Sigma in place of L_eff):

* ``sigma_from_factor`` -- Sigma = L L^T, the sample covariance of Sec. 2.1.
* ``objective_sigma`` / ``gradient_sigma`` -- f(x) = x^T Sigma x + gamma ||x||^2,
  grad f(x) = 2 Sigma x + 2 gamma x.
* ``power_norm2_sigma`` -- the same power method on Sigma: u <- Sigma u /
  ||Sigma u||, returning the Rayleigh quotient u^T Sigma u (= ||L^T u||^2
  when Sigma = L L^T).
* ``npga_sigma`` -- Algorithm 1 with that gradient.

Step-size and momentum variants of Sec. 3.1 (``npga`` / ``npga_sigma``
keywords):

* ``momentum="constant"`` -- the strongly convex specialisation: beta_k
  fixed at (1 - sqrt(alpha m_f)) / (1 + sqrt(alpha m_f)) for a lower
  curvature bound m_f > 0 and a fixed step alpha.
* ``backtrack=(alpha0, rho)`` -- the accelerated backtracking rule: the
  trial step starts at the previous accepted step (alpha0 at k = 0) and is
  multiplied by rho until f(x+) <= f(y) + <grad f(y), x+ - y> +
  ||x+ - y||^2 / (2 alpha); the KKT residual uses the accepted step.
  Reading: f is quadratic, so with d = x+ - y the inequality is exactly
  ||L^T d||^2 + gamma ||d||^2 <= ||d||^2 / (2 alpha) (d^T Sigma d in the
  explicit form).  That form is evaluated: the printed one subtracts
  nearly equal objective values and, near the solution, rejects steps on
  rounding noise alone.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

from .projection import PROJ_OK, project_F


def objective(Leff, gamma, x):
    z = Leff.T @ x
    return float(z @ z + gamma * (x @ x))


def gradient(Leff, gamma, x):
    return 2.0 * (Leff @ (Leff.T @ x)) + 2.0 * gamma * x


def power_norm2(Leff, r, iters: int = 50):
    """Power-method estimate of ||L_eff||_2^2 from the start vector r."""
    u = np.asarray(r, dtype=np.float64)
    u = u / np.linalg.norm(u)
    for _ in range(iters):
        w = Leff @ (Leff.T @ u)
        nw = np.linalg.norm(w)
        if nw == 0.0:
            return 0.0
        u = w / nw
    z = Leff.T @ u
    return float(z @ z)


def _lanczos_top(apply_a, r, steps: int):
    """k-step Lanczos on the symmetric operator apply_a from r; returns the
    largest eigenvalue of the tridiagonal matrix and the steps taken."""
    q = np.asarray(r, dtype=np.float64)
    nr = np.linalg.norm(q)
    if steps < 1 or nr == 0.0:
        return 0.0, 0
    q = q / nr
    q_prev = np.zeros_like(q)
    alphas, betas = [], []
    beta = 0.0
    for _ in range(steps):
        w = apply_a(q)
        a = float(q @ w)
        w = w - a * q - beta * q_prev
        alphas.append(a)
        beta_next = float(np.linalg.norm(w))
        if not beta_next > 1e-12 * (abs(a) + beta):
            break                                   # K_j invariant: the Ritz values are eigenvalues
        betas.append(beta_next)
        q_prev, q, beta = q, w / beta_next, beta_next
    k = len(alphas)
    off = np.array(betas[:k - 1])
    if k == 1:
        return alphas[0], 1
    top = scipy.linalg.eigh_tridiagonal(np.array(alphas), off, eigvals_only=True)[-1]
    return float(top), k


def lanczos_norm2(Leff, r, steps: int = 25):
    """Lanczos estimate of ||L_eff||_2^2 (largest eigenvalue of L L^T) from
    ``steps`` products L(L^T q)."""
    Leff = np.asarray(Leff, dtype=np.float64)
    return _lanczos_top(lambda q: Leff @ (Leff.T @ q), r, steps)[0]


def lanczos_norm2_sigma(Sigma, r, steps: int = 25):
    """The same Lanczos estimate with the explicit Sigma u as the product."""
    Sigma = np.asarray(Sigma, dtype=np.float64)
    return _lanczos_top(lambda q: Sigma @ q, r, steps)[0]


def step_size(lam_hat, gamma, safety: float = 1e-3):
    """alpha = 1 / L_f,  L_f = 2 (lam_hat (1 + safety) + gamma)."""
    return 1.0 / (2.0 * (lam_hat * (1.0 + safety) + gamma))


def kkt_residual(Leff, gamma, mu, R, x, alpha, mode="ge"):
    """||Pi_F(x - alpha grad f(x)) - x||_2 (Sec. 3.1, stopping condition)."""
    p = project_F(x - alpha * gradient(Leff, gamma, x), mu, R, mode)
    return float(np.linalg.norm(p.x - x))


@dataclass
class NPGAResult:
    x: np.ndarray
    iters: int
    kkt: float
    f: float
    converged: bool
    proj_failures: int = 0
    kkt_history: list = field(default_factory=list)
    trajectory: list = field(default_factory=list)   # x^0, x^1, ... if recorded
    alpha: float = 0.0                               # the (last accepted) step


def initial_point(mu, R, mode="ge"):
    """x^0 = Pi_F(1/n 1): a feasible start (the paper only asks x^0 in F)."""
    n = mu.shape[0]
    return project_F(np.full(n, 1.0 / n), mu, R, mode).x


def _npga_loop(fval, grad, curv, gamma, mu, R, x0, alpha, eps, max_iter, kkt_every, mode, record,
               momentum, m_f, backtrack):
    """Algorithm 1 for f with value ``fval``, gradient ``grad`` and curvature
    ``curv(d)`` = f(y + d) - f(y) - <grad f(y), d>."""
    mu = np.asarray(mu, dtype=np.float64)
    x = np.array(x0, dtype=np.float64)
    y = x.copy()
    t = 1.0
    k = 0
    r = np.inf
    hist = []
    fails = 0
    converged = False
    traj = [x.copy()] if record else []
    if backtrack is not None:
        alpha, rho = float(backtrack[0]), float(backtrack[1])
        if not (alpha > 0.0 and 0.0 < rho < 1.0):
            raise ValueError("backtracking needs alpha0 > 0 and 0 < rho < 1")
    if momentum == "constant":
        if not m_f > 0.0:
            raise ValueError("constant momentum needs a lower curvature bound m_f > 0")
        q = np.sqrt(alpha * m_f)
        beta_c = (1.0 - q) / (1.0 + q)
    elif momentum != "fista":
        raise ValueError("momentum is 'fista' or 'constant'")

    def kkt(xk):
        p = project_F(xk - alpha * grad(xk), mu, R, mode)
        return float(np.linalg.norm(p.x - xk))

    while True:
        if kkt_every > 0 and k % kkt_every == 0:
            r = kkt(x)
            hist.append((k, r))
            if r <= eps:
                converged = True
                break
        if k >= max_iter:
            break
        gy = grad(y)
        while True:
            p = project_F(y - alpha * gy, mu, R, mode)
            if backtrack is None:
                break
            d = p.x - y
            if curv(d) <= (d @ d) / (2.0 * alpha):
                break
            alpha *= rho
        if p.status != PROJ_OK:
            fails += 1
        x_new = p.x
        if momentum == "constant":
            beta = beta_c
            t_new = t
        else:
            t_new = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
            beta = (t - 1.0) / t_new
        y = x_new + beta * (x_new - x)
        x, t = x_new, t_new
        k += 1
        if record:
            traj.append(x.copy())
    if not converged:
        r = kkt(x)
    res = NPGAResult(x, k, r, fval(x), converged, fails, hist, traj)
    res.alpha = alpha
    return res


def npga(Leff, gamma, mu, R, x0, alpha, eps=1e-6, max_iter=10000,
         kkt_every=5, mode="ge", record=False, momentum="fista", m_f=0.0,
         backtrack=None) -> NPGAResult:
    """Algorithm 1 on the factor form; a fixed step unless ``backtrack``."""
    Leff = np.asarray(Leff, dtype=np.float64)
    return _npga_loop(lambda x: objective(Leff, gamma, x), lambda x: gradient(Leff, gamma, x),
                      lambda d: objective(Leff, gamma, d), gamma, mu, R, x0, alpha, eps, max_iter, kkt_every,
                      mode, record, momentum, m_f, backtrack)


# ------------------------------------------------------------ explicit Sigma
def sigma_from_factor(L):
    """Sigma = L L^T (Sec. 2.1 with L the centered, 1/sqrt(T-1)-scaled panel)."""
    L = np.asarray(L, dtype=np.float64)
    return L @ L.T


def objective_sigma(Sigma, gamma, x):
    return float(x @ (Sigma @ x) + gamma * (x @ x))


def gradient_sigma(Sigma, gamma, x):
    return 2.0 * (Sigma @ x) + 2.0 * gamma * x


def power_norm2_sigma(Sigma, r, iters: int = 50):
    """Power-method estimate of ||Sigma||_2 (= ||L||_2^2) from the start vector r."""
    u = np.asarray(r, dtype=np.float64)
    u = u / np.linalg.norm(u)
    for _ in range(iters):
        w = Sigma @ u
        nw = np.linalg.norm(w)
        if nw == 0.0:
            return 0.0
        u = w / nw
    return float(u @ (Sigma @ u))


def kkt_residual_sigma(Sigma, gamma, mu, R, x, alpha, mode="ge"):
    p = project_F(x - alpha * gradient_sigma(Sigma, gamma, x), mu, R, mode)
    return float(np.linalg.norm(p.x - x))


def npga_sigma(Sigma, gamma, mu, R, x0, alpha, eps=1e-6, max_iter=10000,
               kkt_every=5, mode="ge", record=False, momentum="fista", m_f=0.0,
               backtrack=None) -> NPGAResult:
    """Algorithm 1 with grad f(y) = 2 Sigma y + 2 gamma y (explicit covariance)."""
    Sigma = np.asarray(Sigma, dtype=np.float64)
    return _npga_loop(lambda x: objective_sigma(Sigma, gamma, x), lambda x: gradient_sigma(Sigma, gamma, x),
                      lambda d: objective_sigma(Sigma, gamma, d), gamma, mu, R, x0, alpha, eps, max_iter,
                      kkt_every, mode, record, momentum, m_f, backtrack)


def vertices_F(mu, R, mode="ge"):
    """Vertex list of F as (i, j, lam): q = lam e_i + (1 - lam) e_j.

    Vertices of the simplex cut by one hyperplane/halfspace are the simplex
    vertices inside F (mu_i >= R; mu_i == R in equality mode) and the points
    where an edge [e_i, e_j] with mu_i > R > mu_j crosses mu^T x = R.
    """
    mu = np.asarray(mu, dtype=np.float64)
    n = mu.shape[0]
    idx = np.arange(n)
    inside = (mu >= R) if mode == "ge" else (mu == R)
    verts = [(int(i), int(i), 1.0) for i in idx[inside]]
    hi = idx[mu > R]
    lo = idx[mu < R]
    for i in hi:
        lam = (R - mu[lo]) / (mu[i] - mu[lo])
        verts.extend((int(i), int(j), float(l)) for j, l in zip(lo, lam))
    return verts


def lin_min_F(g, mu, R, mode="ge"):
    """min_{q in F} <g, q>, exactly, by scanning the vertices of F."""
    g = np.asarray(g, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    inside = (mu >= R) if mode == "ge" else (mu == R)
    best = float(g[inside].min()) if inside.any() else np.inf
    hi = np.nonzero(mu > R)[0]
    lo = np.nonzero(mu < R)[0]
    if hi.size and lo.size:
        for c0 in range(0, hi.size, 256):
            ii = hi[c0:c0 + 256]
            lam = (R - mu[lo][None, :]) / (mu[ii][:, None] - mu[lo][None, :])
            val = lam * g[ii][:, None] + (1.0 - lam) * g[lo][None, :]
            best = min(best, float(val.min()))
    return best


def fw_gap(Leff, gamma, mu, R, x, mode="ge"):
    """Frank--Wolfe gap <grad f(x), x> - min_{q in F} <grad f(x), q>."""
    g = gradient(Leff, gamma, x)
    return float(g @ x) - lin_min_F(g, mu, R, mode)


def solver_gap(f_hat, f_ref):
    """gap_M = max(f_hat - f_ref, 0) / max(|f_ref|, 1e-12) (Sec. 5.2)."""
    return max(f_hat - f_ref, 0.0) / max(abs(f_ref), 1e-12)
