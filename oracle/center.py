"""Sample mean and centered covariance factor (Sec. 2.1) -- test oracle.

For a return panel R (n x T): mu = R 1_T / T, R_c = R - mu 1_T^T and
L = R_c / sqrt(T - 1), so that the unbiased sample covariance is
Sigma = L L^T exactly.  tr(Sigma) = ||L||_F^2.
"""
from __future__ import annotations

import numpy as np


def center_factor(R: np.ndarray):
    """Return (mu, L, trace_sigma) for the n x T panel R, all FP64."""
    R = np.asarray(R, dtype=np.float64)
    n, T = R.shape
    if T < 2:
        raise ValueError("centering needs T >= 2 periods")
    mu = R.sum(axis=1) / T
    L = (R - mu[:, None]) / np.sqrt(T - 1.0)
    trace_sigma = float(np.sum(L * L))
    return mu, L, trace_sigma
