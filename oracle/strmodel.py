"""Sketch--Truncate--Ridge (Sec. 2.5, App. D) -- test oracle, FP64.

* ``sketch``      -- tilde L = L Phi (Sec. 2.3 / 2.5 step 1).  Phi is handed
  in as its transpose (s x T, one sketch column per row).
* ``countsketch_matrix`` / ``countsketch`` -- the sparse map of Sec. 2.3,
  construction (2): Phi(t, h(t)) = s_t, every other entry 0, and
  tilde L = L Phi, i.e. column j of tilde L is the signed sum of the
  columns t of L hashed to j.
* ``truncate``    -- thin SVD of tilde L kept to rank l (Sec. 2.5 step 2),
  computed here from the eigendecomposition of tilde L tilde L^T (n x n):
  its eigenvalues are sigma_i^2 and its eigenvectors are U.  The effective
  factor is L_eff = U_l S_l (n x l), which reproduces
  tilde L_l tilde L_l^T = U_l S_l^2 U_l^T (App. D.3) at O(n l) storage.
* ``ridge_default`` -- gamma = 1e-4 tr(Sigma)/n, the ridge used on the
  compressed workload.
* ``str_covariance`` -- hat Sigma = L_eff L_eff^T + gamma I (Sec. 2.5 step 3).
* ``structured_factor`` -- hat L = [L Phi V_l, sqrt(gamma) I] (App. D.3).
* ``knee_rank`` / ``gamma_for_kappa`` -- the data-driven choices of l and
  gamma of App. D.1 / D.2.
"""
from __future__ import annotations

import numpy as np


def sketch(L, Phi_t):
    return np.asarray(L, dtype=np.float64) @ np.asarray(Phi_t, dtype=np.float64).T


def countsketch_matrix(h, sign, s):
    """Dense T x s matrix Phi with Phi[t, h[t]] = sign[t] (one nonzero per row)."""
    h = np.asarray(h)
    T = h.shape[0]
    Phi = np.zeros((T, s))
    Phi[np.arange(T), h] = np.asarray(sign, dtype=np.float64)
    return Phi


def countsketch(L, h, sign, s):
    """tilde L = L Phi for the CountSketch Phi of (h, sign), in FP64."""
    return np.asarray(L, dtype=np.float64) @ countsketch_matrix(h, sign, s)


def truncate(Ltilde, k):
    """Return (L_eff, sigma, U_k) with L_eff = U_k diag(sigma), sigma descending."""
    Lt = np.asarray(Ltilde, dtype=np.float64)
    K = Lt @ Lt.T
    w, U = np.linalg.eigh(K)
    order = np.argsort(w)[::-1][:k]
    lam = np.maximum(w[order], 0.0)
    sigma = np.sqrt(lam)
    Uk = U[:, order]
    return Uk * sigma[None, :], sigma, Uk


def ridge_default(trace_sigma, n):
    return 1e-4 * float(trace_sigma) / float(n)


def str_covariance(L_eff, gamma):
    L_eff = np.asarray(L_eff, dtype=np.float64)
    return L_eff @ L_eff.T + gamma * np.eye(L_eff.shape[0])


def structured_factor(L, Phi_t, V_l, gamma):
    """hat L = [L Phi V_l, sqrt(gamma) I_n], an n x (l + n) matrix."""
    A = sketch(L, Phi_t) @ V_l
    n = A.shape[0]
    return np.hstack([A, np.sqrt(gamma) * np.eye(n)])


def knee_rank(lam, tau, rho):
    """l = max{i : lam_i/lam_1 >= tau and lam_{i+1}/lam_i <= rho} (App. D.1).

    ``lam`` is sorted nonincreasingly; i is 1-based.  Returns 0 if no index
    qualifies.
    """
    lam = np.asarray(lam, dtype=np.float64)
    best = 0
    for i in range(1, lam.size):        # i = 1 .. r-1 needs lam_{i+1}
        if lam[i - 1] / lam[0] >= tau and lam[i] / lam[i - 1] <= rho:
            best = i
    return best


def gamma_for_kappa(sigma1, kappa_target):
    """gamma = sigma_1^2/(kappa_tar - 1), so kappa(hat Sigma) = kappa_tar (App. D.2)."""
    return float(sigma1) ** 2 / (float(kappa_target) - 1.0)
