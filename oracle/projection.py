"""Projection onto the feasible set F (Sec. 3.1) -- test oracle, FP64.

F = {x : mu^T x >= R, 1^T x = 1, x >= 0} = Delta intersect H.

* ``project_simplex``   -- Eqs. simplex-tau / simplex-proj: sort v in
  descending order, take the largest j with v_j - (sum_{i<=j} v_i - 1)/j > 0,
  tau = (sum_{i<=j} v_i - 1)/j, x = max(v - tau, 0).
* ``project_halfspace`` -- Eq. proj-halfspace (closed form).
* ``project_F``         -- Eq. projF-dualpath: x(nu) = Pi_Delta(v + nu mu),
  phi(nu) = mu^T x(nu) nondecreasing.  If mu^T Pi_Delta(v) >= R the simplex
  projection is already the answer (nu = 0).  Otherwise nu is bracketed by
  geometric expansion nu = 1, 2, 4, ... until phi(nu) >= R, then bisected.
  Reading taken where the paper stops bisection at a residual tolerance: the
  bisection runs until both bracket ends share one support S, and the answer
  is then finished exactly on S by solving the two linear equations
      |S| tau - nu sum_S mu   = sum_S v - 1
      sum_S mu tau - nu sum_S mu^2 = sum_S mu v - R
  and re-verifying x_S > 0 and v_i + nu mu_i - tau <= 0 off S.
  An equality mode (mu^T x = R, nu of either sign) is also provided.
* ``project_F_dykstra`` -- the safeguard of Sec. 3.1: Dykstra's alternating
  projections between Delta and H (Bauschke--Borwein), with the correction
  terms p (for Delta) and q (for H); converges to Pi_F(v).
* ``project_F_safeguarded`` -- the scalar search with a bracketing budget,
  falling back to Dykstra when the bracketing does not close within it.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

PROJ_OK = 0
PROJ_INFEASIBLE = 1
PROJ_TOLERANCE = 2      # bisection stalled; returned x(nu_hi) unverified
PROJ_BRACKET = 3        # the bracketing budget ran out before phi(nu) crossed R


@dataclass
class ProjResult:
    x: np.ndarray
    nu: float
    tau: float
    support: int
    status: int
    residual: float      # mu^T x - R (0 when the return row is inactive)
    active: bool         # return constraint active (nu != 0)


def project_simplex(w: np.ndarray):
    """Euclidean projection onto the unit simplex by sorting (Eq. simplex-tau).

    Returns (x, tau).
    """
    w = np.asarray(w, dtype=np.float64)
    n = w.shape[0]
    u = np.sort(w)[::-1]
    c = np.cumsum(u) - 1.0
    j = np.arange(1, n + 1, dtype=np.float64)
    ok = np.nonzero(u - c / j > 0.0)[0]
    rho = ok[-1]
    tau = c[rho] / (rho + 1.0)
    return np.maximum(w - tau, 0.0), float(tau)


def project_halfspace(y: np.ndarray, mu: np.ndarray, R: float) -> np.ndarray:
    """Projection onto H = {x : mu^T x >= R} (Eq. proj-halfspace)."""
    y = np.asarray(y, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    d = float(mu @ y)
    if d >= R:
        return y.copy()
    return y + (R - d) / float(mu @ mu) * mu


def _x_of_nu(v, mu, nu):
    return project_simplex(v + nu * mu)


def _finish_on_support(v, mu, R, S, lo, hi):
    """Exact (tau, nu) on a fixed support S; None if it does not verify."""
    vs, ms = v[S], mu[S]
    k = float(S.sum())
    if k == 0:
        return None
    sm, smm, sv, smv = ms.sum(), (ms * ms).sum(), vs.sum(), (ms * vs).sum()
    det = -k * smm + sm * sm
    scale = max(1.0, k * smm)
    if abs(det) <= 1e-14 * scale:
        # mu is constant on S: phi is flat on this piece; x_S does not depend on nu.
        nu = 0.5 * (lo + hi)
        tau = (sv + nu * sm - 1.0) / k
    else:
        # Cramer's rule on [[k, -sm], [sm, -smm]] [tau, nu]^T = [sv - 1, smv - R].
        b1, b2 = sv - 1.0, smv - R
        tau = (b1 * (-smm) - (-sm) * b2) / det
        nu = (k * b2 - sm * b1) / det
    w = v + nu * mu - tau
    delta = 1e-12 * max(1.0, float(np.max(np.abs(v + nu * mu))))
    if np.any(w[S] < -delta) or np.any(w[~S] > delta):
        return None
    x = np.where(S, np.maximum(w, 0.0), 0.0)
    return x, float(nu), float(tau)


def project_F(v, mu, R, mode: str = "ge", max_bracket: int = 200,
              max_bisect: int = 2000) -> ProjResult:
    """Exact projection of v onto F (Eq. projF-dualpath) in FP64.

    mode "ge": F uses mu^T x >= R (the paper's set).  mode "eq": mu^T x = R.
    """
    v = np.asarray(v, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    n = v.shape[0]
    if n == 0:
        raise ValueError("empty problem")
    R = float(R)
    if R > mu.max() or (mode == "eq" and R < mu.min()):
        return ProjResult(np.full(n, np.nan), np.nan, np.nan, 0, PROJ_INFEASIBLE, np.nan, False)

    x0, tau0 = project_simplex(v)
    phi0 = float(mu @ x0)
    if phi0 >= R and (mode == "ge" or phi0 == R):
        return ProjResult(x0, 0.0, tau0, int((x0 > 0).sum()), PROJ_OK,
                          phi0 - R if mode == "eq" else 0.0, False)
    sign = 1.0 if phi0 < R else -1.0   # direction in which nu must move

    def far_side(nu):
        x, _ = _x_of_nu(v, mu, nu)
        return sign * (float(mu @ x) - R) >= 0.0

    # Geometric bracketing nu = 1, 2, 4, ... (Sec. 3.1).
    lo, hi = 0.0, sign * 1.0
    for _ in range(max_bracket):
        if far_side(hi):
            break
        lo, hi = hi, 2.0 * hi
    else:
        return ProjResult(np.full(n, np.nan), np.nan, np.nan, 0, PROJ_BRACKET, np.nan, True)

    # Bisection until the support is pinned, then the exact finish.
    for _ in range(max_bisect):
        xl, _ = _x_of_nu(v, mu, lo)
        xh, _ = _x_of_nu(v, mu, hi)
        Sl, Sh = xl > 0.0, xh > 0.0
        for S in ((Sl,) if np.array_equal(Sl, Sh) else (Sl, Sh)):
            got = _finish_on_support(v, mu, R, S, min(lo, hi), max(lo, hi))
            if got is not None:
                x, nu, tau = got
                return ProjResult(x, nu, tau, int((x > 0).sum()), PROJ_OK,
                                  float(mu @ x) - R, True)
        mid = 0.5 * (lo + hi)
        if mid == lo or mid == hi:
            break
        if far_side(mid):
            hi = mid
        else:
            lo = mid
    x, tau = _x_of_nu(v, mu, hi)
    return ProjResult(x, float(hi), tau, int((x > 0).sum()), PROJ_TOLERANCE,
                      float(mu @ x) - R, True)


def active_set(v, mu, nu, tau, rel_degenerate: float = 1e-12):
    """Active-set indicator (v_i + nu mu_i - tau > 0) and a degeneracy mask.

    Entries within rel_degenerate * max|v| of the threshold are flagged as
    degenerate; the active-set identity is only meaningful off that mask.
    """
    v = np.asarray(v, dtype=np.float64)
    w = v + nu * np.asarray(mu, dtype=np.float64) - tau
    tol = rel_degenerate * max(1.0, float(np.max(np.abs(v))))
    return w > 0.0, np.abs(w) <= tol


def project_hyperplane(y: np.ndarray, mu: np.ndarray, R: float) -> np.ndarray:
    """Projection onto {x : mu^T x = R}."""
    y = np.asarray(y, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    return y + (R - float(mu @ y)) / float(mu @ mu) * mu


def project_F_dykstra(v, mu, R, mode: str = "ge", iters: int = 100000, tol: float = 1e-13):
    """Dykstra's algorithm for Pi_{Delta cap H}(v) (Sec. 3.1 safeguard).

    x^0 = v, p^0 = q^0 = 0;  y = Pi_Delta(x + p), p <- x + p - y;
    x = Pi_H(y + q), q <- y + q - x.  Stops at a fixed point of the whole
    state (x, p, q): a sweep that moves none of them by more than
    tol * max(1, |v|_inf), with x and y in agreement.  (x alone can stand
    still for many sweeps while the corrections still move.)  Returns
    (x, sweeps).
    """
    v = np.asarray(v, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    proj_H = (lambda w: project_halfspace(w, mu, R)) if mode == "ge" else (lambda w: project_hyperplane(w, mu, R))
    x = v.copy()
    p = np.zeros_like(v)
    q = np.zeros_like(v)
    scale = tol * max(1.0, float(np.max(np.abs(v))))
    for it in range(1, iters + 1):
        y, _ = project_simplex(x + p)
        p_new = x + p - y
        x_new = proj_H(y + q)
        q_new = y + q - x_new
        moved = max(float(np.max(np.abs(x_new - x))), float(np.max(np.abs(p_new - p))),
                    float(np.max(np.abs(q_new - q))))
        x, p, q = x_new, p_new, q_new
        if moved <= scale and float(np.max(np.abs(x - y))) <= scale:
            return y, it
    return y, iters


def project_F_safeguarded(v, mu, R, mode: str = "ge", max_bracket: int = 200,
                          dykstra_iters: int = 100000) -> ProjResult:
    """The scalar-search projection; Dykstra when its bracketing budget runs out."""
    res = project_F(v, mu, R, mode, max_bracket=max_bracket)
    if res.status != PROJ_BRACKET:
        return res
    x, _ = project_F_dykstra(v, mu, R, mode, dykstra_iters)
    return ProjResult(x, np.nan, np.nan, int((x > 0).sum()), PROJ_OK, float(np.asarray(mu) @ x) - R, True)
