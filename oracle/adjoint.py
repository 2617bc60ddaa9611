"""Reverse-mode derivative of the unrolled NPGA solve -- test oracle, FP64.

The paper does not differentiate its solver; these are the conventions used
here (stated so the CUDA adjoint can be checked against them):

* The solve is Algorithm 1 unrolled for exactly K iterations with a fixed
  step alpha and start x^0; alpha, x^0 and the target R are constants (no
  derivative flows through the power method or the choice of R).
* Iteration k: z_k = L^T y_k, v_k = y_k - alpha (2 L z_k + 2 gamma y_k),
  x_{k+1} = Pi_F(v_k; mu, R), y_{k+1} = x_{k+1} + beta_k (x_{k+1} - x_k).
  The output is x_K.
* Projection derivative on the support S of x_{k+1} with the tight rows
  C = [1_S, mu_S] (or [1_S] when the return row is slack): x_S = P v_S + ...,
  P = I - C (C^T C)^{-1} C^T, zero off S.  With a = adjoint of x_{k+1} and
  c = (C^T C)^{-1} C^T a_S:  v_bar = P a (on S), and
  mu_bar += nu P a - x c_mu (on S; zero when the return row is slack).
* v = y - alpha (2 L L^T y + 2 gamma y) gives
  y_bar = v_bar - alpha (2 L L^T v_bar + 2 gamma v_bar) and
  L_bar += -2 alpha (v_bar z_k^T + y_k (L^T v_bar)^T).

``grad_check_directions`` returns central finite differences of the loss
along given directions, computed with the FP64 forward.
"""
from __future__ import annotations

import numpy as np

from .projection import project_F


def fista_betas(K):
    """beta_k = (t_k - 1)/t_{k+1} with t_0 = 1 (Algorithm 1)."""
    t = 1.0
    out = []
    for _ in range(K):
        tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        out.append((t - 1.0) / tn)
        t = tn
    return out


def unrolled_forward(L, gamma, mu, R, x0, alpha, K, mode="ge", record=False):
    """x_K of K NPGA iterations; optionally the tape needed by ``backward``."""
    L = np.asarray(L, dtype=np.float64)
    x = np.array(x0, dtype=np.float64)
    y = x.copy()
    betas = fista_betas(K)
    tape = []
    for k in range(K):
        z = L.T @ y
        v = y - alpha * (2.0 * (L @ z) + 2.0 * gamma * y)
        p = project_F(v, mu, R, mode)
        xn = p.x
        if record:
            tape.append({"y": y, "z": z, "x1": xn, "nu": p.nu, "active": p.active or mode == "eq"})
        y = xn + betas[k] * (xn - x)
        x = xn
    return (x, tape, betas) if record else x


def backward(L, gamma, mu, alpha, tape, betas, xbar_K):
    """(mu_bar, L_bar) for the loss gradient xbar_K = d loss / d x_K."""
    L = np.asarray(L, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    n = L.shape[0]
    xbar = np.array(xbar_K, dtype=np.float64)
    ybar = np.zeros(n)
    mubar = np.zeros(n)
    Lbar = np.zeros_like(L)
    for k in range(len(tape) - 1, -1, -1):
        rec = tape[k]
        a = xbar + (1.0 + betas[k]) * ybar
        xbar = -betas[k] * ybar
        S = rec["x1"] > 0.0
        if rec["active"]:
            C = np.stack([np.ones(S.sum()), mu[S]], axis=1)
        else:
            C = np.ones((S.sum(), 1))
        c = np.linalg.solve(C.T @ C, C.T @ a[S])
        vbar = np.zeros(n)
        vbar[S] = a[S] - C @ c
        if rec["active"]:
            mubar[S] += rec["nu"] * vbar[S] - rec["x1"][S] * c[1]
        w = L.T @ vbar
        ybar = vbar - alpha * (2.0 * (L @ w) + 2.0 * gamma * vbar)
        Lbar += -2.0 * alpha * (np.outer(vbar, rec["z"]) + np.outer(rec["y"], w))
    return mubar, Lbar


def sharpe_loss(x, mu_test, L_test):
    """-(mu_test^T x) / sqrt(x^T Sigma_test x), Sigma_test = L_test L_test^T."""
    s = np.linalg.norm(L_test.T @ x)
    return -(mu_test @ x) / s


def sharpe_loss_grad(x, mu_test, L_test):
    q = L_test @ (L_test.T @ x)
    s = np.sqrt(x @ q)
    return -mu_test / s + (mu_test @ x) * q / s ** 3


def grad_check_directions(L, gamma, mu, R, x0, alpha, K, loss, dirs_mu, dirs_L, h=1e-4, mode="ge"):
    """Central differences of loss(x_K(mu + h d_mu, L + h d_L)) along each direction pair."""
    out = []
    for dm, dL in zip(dirs_mu, dirs_L):
        fp = loss(unrolled_forward(L + h * dL, gamma, mu + h * dm, R, x0, alpha, K, mode))
        fm = loss(unrolled_forward(L - h * dL, gamma, mu - h * dm, R, x0, alpha, K, mode))
        out.append((fp - fm) / (2.0 * h))
    return np.array(out)
