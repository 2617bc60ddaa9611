"""Exhaustive enumeration for tiny problems (n <= 10) -- test oracle, FP64.

Both functions rest on one fact about a convex problem over the polytope F:
its solution lies in the relative interior of some face, and is therefore the
minimiser of the same objective over that face's affine hull.  Faces of F are
indexed by a support S (x_i = 0 off S) and by whether the return row
mu^T x = R is tight.  Enumerating every (S, tight) pair, solving the
equality-constrained problem on it and keeping the best candidate that lies
in F gives the exact answer with no iteration and no tolerance choice.

* ``project_bruteforce`` -- argmin ||x - v|| over F.
* ``qp_bruteforce``      -- argmin x^T Sigma x over F (Sigma positive definite).
"""
from __future__ import annotations

import itertools

import numpy as np


def _faces(n, mode):
    for size in range(1, n + 1):
        for S in itertools.combinations(range(n), size):
            for tight in ((False, True) if mode == "ge" else (True,)):
                yield np.array(S), tight


def _constraints(mu, S, tight, R):
    rows = [np.ones(S.size)]
    rhs = [1.0]
    if tight:
        rows.append(mu[S])
        rhs.append(R)
    return np.array(rows), np.array(rhs)


def _in_F(x, mu, R, mode, tol):
    if np.any(x < -tol) or abs(x.sum() - 1.0) > tol:
        return False
    r = mu @ x - R
    return r >= -tol if mode == "ge" else abs(r) <= tol


def project_bruteforce(v, mu, R, mode="ge", tol=1e-12):
    v = np.asarray(v, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    n = v.size
    if n > 12:
        raise ValueError("brute force is for tiny n only")
    best, best_d = None, np.inf
    for S, tight in _faces(n, mode):
        C, d = _constraints(mu, S, tight, R)
        # x_S = v_S - C^T lam with (C C^T) lam = C v_S - d.
        lam = np.linalg.lstsq(C @ C.T, C @ v[S] - d, rcond=None)[0]
        xs = v[S] - C.T @ lam
        if np.max(np.abs(C @ xs - d)) > 1e-10:
            continue   # inconsistent face (e.g. mu constant on S, != R)
        x = np.zeros(n)
        x[S] = xs
        if not _in_F(x, mu, R, mode, tol):
            continue
        dist = float(np.sum((x - v) ** 2))
        if dist < best_d - 1e-15:
            best, best_d = x, dist
    return best


def qp_bruteforce(Sigma, mu, R, mode="ge", tol=1e-12):
    Sigma = np.asarray(Sigma, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    n = mu.size
    if n > 12:
        raise ValueError("brute force is for tiny n only")
    best, best_f = None, np.inf
    for S, tight in _faces(n, mode):
        C, d = _constraints(mu, S, tight, R)
        m = C.shape[0]
        K = np.zeros((S.size + m, S.size + m))
        K[:S.size, :S.size] = 2.0 * Sigma[np.ix_(S, S)]
        K[:S.size, S.size:] = C.T
        K[S.size:, :S.size] = C
        rhs = np.concatenate([np.zeros(S.size), d])
        sol = np.linalg.lstsq(K, rhs, rcond=None)[0]
        xs = sol[:S.size]
        if np.max(np.abs(C @ xs - d)) > 1e-10:
            continue
        x = np.zeros(n)
        x[S] = xs
        if not _in_F(x, mu, R, mode, tol):
            continue
        f = float(x @ Sigma @ x)
        if f < best_f - 1e-18:
            best, best_f = x, f
    return best
