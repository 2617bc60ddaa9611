"""NPGA (Algorithm 1) and its certificates -- test oracle, FP64.

* ``objective`` / ``gradient`` -- Eq. npga-unified-grad:
  f(x) = ||L_eff^T x||^2 + gamma ||x||^2,  grad f(x) = 2 L_eff (L_eff^T x) + 2 gamma x.
* ``power_norm2`` -- the power method of the Sec. 3.1 remark:
  u <- L(L^T u)/||L(L^T u)||, u^0 = r/||r||; returns ||L^T u||^2, an
  estimate of ||L_eff||_2^2.
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
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

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


def initial_point(mu, R, mode="ge"):
    """x^0 = Pi_F(1/n 1): a feasible start (the paper only asks x^0 in F)."""
    n = mu.shape[0]
    return project_F(np.full(n, 1.0 / n), mu, R, mode).x


def npga(Leff, gamma, mu, R, x0, alpha, eps=1e-6, max_iter=10000,
         kkt_every=5, mode="ge", record=False) -> NPGAResult:
    """Algorithm 1 with a fixed step (every benchmark in the paper uses one)."""
    Leff = np.asarray(Leff, dtype=np.float64)
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
    while True:
        if kkt_every > 0 and k % kkt_every == 0:
            r = kkt_residual(Leff, gamma, mu, R, x, alpha, mode)
            hist.append((k, r))
            if r <= eps:
                converged = True
                break
        if k >= max_iter:
            break
        v = y - alpha * gradient(Leff, gamma, y)
        p = project_F(v, mu, R, mode)
        if p.status != PROJ_OK:
            fails += 1
        x_new = p.x
        t_new = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        beta = (t - 1.0) / t_new
        y = x_new + beta * (x_new - x)
        x, t = x_new, t_new
        k += 1
        if record:
            traj.append(x.copy())
    if not converged:
        r = kkt_residual(Leff, gamma, mu, R, x, alpha, mode)
    return NPGAResult(x, k, r, objective(Leff, gamma, x), converged, fails, hist, traj)


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
