"""Pins of the FP64 oracle adjoint (oracle/adjoint.py): directional
derivatives of a loss on the unrolled NPGA output against central finite
differences of the FP64 forward, direction by direction, skipping
directions whose +-h forwards change an active set along the path (kinks)."""
import numpy as np
import pytest

from synth import CFG_SMALL, factor_returns
from oracle.center import center_factor
from oracle.npga import initial_point, power_norm2, step_size
from oracle import adjoint
from synth import power_start


def supports(L, gamma, mu, R, x0, alpha, K, mode):
    _, tape, _ = adjoint.unrolled_forward(L, gamma, mu, R, x0, alpha, K, mode, record=True)
    return [tuple(np.nonzero(r["x1"] > 0)[0]) + (r["active"],) for r in tape]


@pytest.mark.parametrize("mode,gamma", [("ge", 0.0), ("ge", 3e-5), ("eq", 0.0)])
def test_adjoint_matches_finite_differences(mode, gamma):
    n, T, Ttest, K = 10, 40, 30, 25
    R = factor_returns(CFG_SMALL.scaled(n, T + Ttest, seed=71), np.float32).astype(np.float64)
    mu, L, _ = center_factor(R[:, :T])
    mu_t, L_t, _ = center_factor(R[:, T:])
    Rt = float(np.percentile(mu, 70))
    alpha = step_size(power_norm2(L, power_start(n), 100), gamma)
    x0 = initial_point(mu, Rt, mode)
    loss = lambda x: adjoint.sharpe_loss(x, mu_t, L_t)
    xK, tape, betas = adjoint.unrolled_forward(L, gamma, mu, Rt, x0, alpha, K, mode, record=True)
    gx = adjoint.sharpe_loss_grad(xK, mu_t, L_t)
    # the loss gradient itself against finite differences
    e = np.random.default_rng(0).standard_normal(n) * 1e-3
    fd = (loss(xK + 1e-4 * e) - loss(xK - 1e-4 * e)) / 2e-4
    assert gx @ e == pytest.approx(fd, rel=1e-6)
    mub, Lb = adjoint.backward(L, gamma, mu, alpha, tape, betas, gx)
    rng = np.random.default_rng(1)
    base = supports(L, gamma, mu, Rt, x0, alpha, K, mode)
    h = 1e-6
    checked = 0
    for _ in range(12):
        dm = rng.standard_normal(n)
        dm *= np.sqrt(np.mean(mu ** 2)) / np.linalg.norm(dm)
        dL = rng.standard_normal(L.shape)
        dL *= np.sqrt(np.mean(L ** 2)) / np.linalg.norm(dL)
        if (supports(L + h * dL, gamma, mu + h * dm, Rt, x0, alpha, K, mode) != base or
                supports(L - h * dL, gamma, mu - h * dm, Rt, x0, alpha, K, mode) != base):
            continue                                   # a kink along the path: FD is not a derivative
        fd = adjoint.grad_check_directions(L, gamma, mu, Rt, x0, alpha, K, loss, [dm], [dL], h=h, mode=mode)[0]
        an = mub @ dm + np.sum(Lb * dL)
        assert an == pytest.approx(fd, rel=2e-5, abs=1e-9 * abs(fd) + 1e-12)
        checked += 1
    assert checked >= 8
