"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module draws random numbers and nothing else: it holds none of the
method's arithmetic (no centering, no covariance, no projection).  Both the
oracle under ``oracle/`` and the GPU binding take their inputs from here, so
that the two sides see bit-identical data.

Workloads (the paper's data is a proprietary 5-minute A-share panel, so a
seeded factor model of the same shape stands in for it, Sec. 5.2):

* ``factor_returns`` -- R = B f + eps + drift 1^T, with Gaussian loadings B,
  Student-t(4) factors scaled to a target per-period volatility, Gaussian
  idiosyncratic noise with per-asset volatility drawn uniformly, and a
  per-asset drift drawn uniformly.  Draw order is fixed (B, f, sigma, eps,
  drift) on one NumPy PCG64 stream so that a seed names one panel.
* ``power_start`` -- the random start r ~ N(0, I_n) of the power method
  (Sec. 3.1, remark on the power method); the method normalises it.
* ``gaussian_sketch`` -- the JL sketch Phi with i.i.d. N(0, 1/s) entries
  (Sec. 2.3), stored column by column (one sketch column is contiguous).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "factor_returns_device",
    "FactorModel",
    "CFG_SMALL",
    "CFG_FULL",
    "factor_returns",
    "power_start",
    "gaussian_sketch",
    "uneven_problem_sizes",
]


@dataclass(frozen=True)
class FactorModel:
    """Recipe of a synthetic return panel (shape, seed and distributions)."""

    n: int                      # assets
    T: int                      # periods
    n_factors: int
    seed: int
    idio_lo: float              # idiosyncratic vol ~ U(idio_lo, idio_hi)
    idio_hi: float
    drift_lo: float = -2e-4     # per-asset drift ~ U(drift_lo, drift_hi)
    drift_hi: float = 6e-4
    loading_scale: float = 0.01  # B ~ N(0,1) * loading_scale
    factor_vol: float = 0.01     # per-period vol of each Student-t factor
    t_dof: float = 4.0

    def scaled(self, n: int, T: int, seed: int | None = None) -> "FactorModel":
        """Same distributions at another shape (used for reduced test sizes)."""
        return FactorModel(n, T, self.n_factors, self.seed if seed is None else seed,
                           self.idio_lo, self.idio_hi, self.drift_lo, self.drift_hi,
                           self.loading_scale, self.factor_vol, self.t_dof)


# 200 assets x 1000 periods, 5 factors, idiosyncratic vol 0.5%..2%, seed 0.
CFG_SMALL = FactorModel(n=200, T=1000, n_factors=5, seed=0, idio_lo=0.005, idio_hi=0.02)
# The paper's real-data shape: 5440 assets x 48374 training periods,
# 20 factors, idiosyncratic vol 1%..3%, seed 1.
CFG_FULL = FactorModel(n=5440, T=48374, n_factors=20, seed=1, idio_lo=0.01, idio_hi=0.03)


def factor_returns(model: FactorModel, dtype=np.float64) -> np.ndarray:
    """Return the n x T return panel R (row i = asset i), C-contiguous.

    The panel is drawn in FP64; ``dtype=np.float32`` rounds it once at the
    end (the GPU path stores FP32, and the oracle is then handed the same
    rounded values widened back to FP64).
    """
    rng = np.random.default_rng(model.seed)
    n, T, k = model.n, model.T, model.n_factors
    B = rng.standard_normal((n, k)) * model.loading_scale
    # Student-t with nu dof has variance nu/(nu-2); rescale to factor_vol.
    t_scale = model.factor_vol / math.sqrt(model.t_dof / (model.t_dof - 2.0))
    f = rng.standard_t(model.t_dof, size=(k, T)) * t_scale
    sig = rng.uniform(model.idio_lo, model.idio_hi, size=n)
    R = np.empty((n, T), dtype=np.float64)
    # Fill row blocks to bound the temporary footprint at full size.
    blk = max(1, (1 << 24) // max(T, 1))
    for i0 in range(0, n, blk):
        i1 = min(n, i0 + blk)
        R[i0:i1] = rng.standard_normal((i1 - i0, T))
        R[i0:i1] *= sig[i0:i1, None]
    drift = rng.uniform(model.drift_lo, model.drift_hi, size=n)
    for i0 in range(0, n, blk):
        i1 = min(n, i0 + blk)
        R[i0:i1] += B[i0:i1] @ f
        R[i0:i1] += drift[i0:i1, None]
    if dtype == np.float64:
        return R
    return R.astype(dtype)


def power_start(n: int, seed: int = 7) -> np.ndarray:
    """Unnormalised start vector r ~ N(0, I_n) of the power method."""
    return np.random.default_rng(seed).standard_normal(n)


def gaussian_sketch(T: int, s: int, seed: int = 2, dtype=np.float64) -> np.ndarray:
    """JL sketch with i.i.d. N(0, 1/s) entries, returned as an s x T array.

    Row j of the result is column j of Phi (T x s), so each sketch column is
    contiguous -- the layout the sketch GEMM consumes.
    """
    rng = np.random.default_rng(seed)
    out = np.empty((s, T), dtype=dtype)
    scale = 1.0 / math.sqrt(s)
    blk = max(1, (1 << 24) // max(T, 1))
    for j0 in range(0, s, blk):
        j1 = min(s, j0 + blk)
        out[j0:j1] = rng.standard_normal((j1 - j0, T)) * scale
    return out


def countsketch_hash(T: int, s: int, seed: int = 2):
    """The random draws of a CountSketch map (Sec. 2.3, construction (2)):
    bucket h(t) uniform in [0, s) and sign s_t uniform in {-1, +1} for each
    period t.  Returns (h int32 [T], sign int8 [T])."""
    rng = np.random.default_rng(seed)
    h = rng.integers(0, s, size=T, dtype=np.int64).astype(np.int32)
    sign = (2 * rng.integers(0, 2, size=T, dtype=np.int64) - 1).astype(np.int8)
    return h, sign


def uneven_problem_sizes(count: int = 256, seed: int = 1000,
                         n_range=(500, 5000), T_range=(2000, 20000)):
    """Shapes of a batch of independent problems of uneven size.

    Problem j has n_j ~ U[n_range] and T_j ~ U[T_range] (integers, drawn from
    seed ``seed``); its panel is ``factor_returns`` of the small-config
    distributions with seed ``seed + j``.
    """
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_range[0], n_range[1] + 1, size=count)
    Ts = rng.integers(T_range[0], T_range[1] + 1, size=count)
    return [CFG_SMALL.scaled(int(a), int(b), seed=seed + j) for j, (a, b) in enumerate(zip(ns, Ts))]


def factor_returns_device(model: FactorModel, device="cuda", dtype=None):
    """The same factor-model distributions drawn on the GPU with PyTorch's
    seeded generator (a different random stream from ``factor_returns``).

    Used where drawing billions of numbers on the host would dominate a
    measurement (the 256-problem uneven batch); parity tests use the NumPy
    stream so that the oracle sees identical inputs.  Returns an n x T FP32
    tensor.
    """
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(model.seed))
    n, T, k = model.n, model.T, model.n_factors
    f32 = torch.float32
    B = torch.randn((n, k), generator=g, device=device, dtype=f32) * model.loading_scale
    # Student-t(nu) = N(0,1) / sqrt(chi2(nu)/nu); chi2 via a sum of squared normals
    nrm = torch.randn((k, T), generator=g, device=device, dtype=f32)
    chi = torch.randn((int(model.t_dof), k, T), generator=g, device=device, dtype=f32).pow_(2).sum(0)
    t = nrm / torch.sqrt(chi / model.t_dof)
    f = t * (model.factor_vol / math.sqrt(model.t_dof / (model.t_dof - 2.0)))
    sig = torch.rand(n, generator=g, device=device, dtype=f32) * (model.idio_hi - model.idio_lo) + model.idio_lo
    R = torch.randn((n, T), generator=g, device=device, dtype=f32) * sig[:, None]
    drift = torch.rand(n, generator=g, device=device, dtype=f32) * (model.drift_hi - model.drift_lo) + model.drift_lo
    R += B @ f
    R += drift[:, None]
    return R
