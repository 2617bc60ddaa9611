"""GPU parity of the step and momentum variants of Sec. 3.1 and of the
Dykstra safeguard of the projection.

* Constant momentum (strongly convex specialisation): beta fixed at
  (1 - sqrt(alpha m_f)) / (1 + sqrt(alpha m_f)) with m_f = 2 gamma; the
  solution matches the oracle's run of the same rule (and hence x*) within
  1e-4, and the stopping iteration agrees with the oracle's to within two
  KKT periods.
* Backtracking: from a trial step 100x the power-method step, the accepted
  step lies in [rho / L_f, alpha0], at least one trial was rejected, and the
  solution matches the oracle's backtracking run within 1e-4 -- on the
  fused single pass, the two-pass kernels and the explicit-Sigma product.
* Dykstra safeguard: with a one-step budget for the scalar search the
  safeguard takes over (info["dykstra"] > 0) and the solve still converges
  to the oracle's point; without it the same budget leaves failed
  projections.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import CFG_FULL, factor_returns, power_start
from oracle.npga import initial_point, npga, npga_sigma, objective, power_norm2, step_size

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def mv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02917_gb300 import mv as m
    m.lib()
    return m


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def problem(mv, n, T, seed, pct=60, layout="nt"):
    R = gpu(factor_returns(CFG_FULL.scaled(n, T, seed=seed), np.float32))
    L, _, mu, _ = mv.center_factor(R, "f32", layout=layout)
    if layout == "tn":
        Lq = L[:T, :n].double().cpu().numpy().T
    else:
        Lq = L[:, :T].double().cpu().numpy()
    mu_o = mu.cpu().numpy()
    return L, mu, Lq, mu_o, float(np.percentile(mu_o, pct))


@pytest.mark.parametrize("gamma", [5e-5, 2e-4])
def test_constant_momentum_parity(mv, gamma):
    n, T = 700, 3000
    L, mu, Lq, mu_o, Rt = problem(mv, n, T, seed=51)
    r0 = power_start(n)
    x, info = mv.npga_solve(L, mu, Rt, T, gamma=gamma, eps=1e-6, power_start=gpu(r0), momentum=1)
    assert info["converged"] == 1 and info["kkt"] <= 1e-6
    lam = power_norm2(Lq, r0, 50)
    a = step_size(lam, gamma)
    assert info["alpha"] == pytest.approx(a, rel=1e-5)
    ref = npga(Lq, gamma, mu_o, Rt, initial_point(mu_o, Rt), a, eps=1e-6, max_iter=100000,
               momentum="constant", m_f=2 * gamma)
    assert ref.converged
    assert abs(info["iterations"] - ref.iters) <= 10
    exact = npga(Lq, gamma, mu_o, Rt, initial_point(mu_o, Rt), a, eps=1e-11, max_iter=200000)
    assert np.max(np.abs(x.cpu().numpy() - exact.x)) <= 1e-4
    # objective from the kept L L^T x of the last KKT test
    assert info["objective"] == pytest.approx(objective(Lq, gamma, x.cpu().numpy()), rel=1e-5)
    # the FISTA run of the same problem lands on the same point
    xf, _ = mv.npga_solve(L, mu, Rt, T, gamma=gamma, eps=1e-6, power_start=gpu(r0))
    assert np.max(np.abs(xf.cpu().numpy() - x.cpu().numpy())) <= 2e-4


@pytest.mark.parametrize("path", ["fused_tn", "two_pass", "sigma"])
def test_backtracking_parity(mv, path):
    n, T = 1100, 4500
    layout = "tn" if path == "fused_tn" else "nt"
    L, mu, Lq, mu_o, Rt = problem(mv, n, T, seed=53, layout=layout)
    r0 = power_start(n)
    lam = power_norm2(Lq, r0, 50)
    a_pow = step_size(lam, 0.0)
    Lf = 2.0 * np.linalg.eigvalsh(Lq @ Lq.T)[-1]
    a0, rho = 100.0 * a_pow, 0.5
    kw = dict(eps=1e-6, power_start=gpu(r0), backtrack=1, bt_alpha0=a0, bt_rho=rho)
    if path == "sigma":
        S = mv.sigma_form(L, T, "f32")
        x, info = mv.npga_solve(S, mu, Rt, T, layout="sigma", **kw)
    else:
        x, info = mv.npga_solve(L, mu, Rt, T, layout=layout, two_pass=1 if path == "two_pass" else 0, **kw)
    assert info["converged"] == 1 and info["kkt"] <= 1e-6
    assert info["backtracks"] >= 1
    assert rho / Lf * (1 - 1e-6) <= info["alpha"] <= a0
    ref = npga(Lq, 0.0, mu_o, Rt, initial_point(mu_o, Rt), 0.0, eps=1e-11, max_iter=200000,
               backtrack=(a0, rho))
    assert ref.converged
    assert np.max(np.abs(x.cpu().numpy() - ref.x)) <= 1e-4
    # objective by one more product at the returned x (the backtracking path)
    assert info["objective"] == pytest.approx(objective(Lq, 0.0, x.cpu().numpy()), rel=1e-5)


def test_backtracking_default_trial_and_constant_momentum(mv):
    """Trial step = power-method step / rho^4 by default; both variants at once."""
    n, T, gamma = 600, 2500, 1e-4
    L, mu, Lq, mu_o, Rt = problem(mv, n, T, seed=57)
    r0 = power_start(n)
    x, info = mv.npga_solve(L, mu, Rt, T, gamma=gamma, eps=1e-6, power_start=gpu(r0), backtrack=1, momentum=1)
    assert info["converged"] == 1
    lam = power_norm2(Lq, r0, 50)
    assert info["alpha"] <= step_size(lam, gamma, 0.0) / 0.5 ** 4 * (1 + 1e-9)
    exact = npga(Lq, gamma, mu_o, Rt, initial_point(mu_o, Rt), step_size(lam, gamma), eps=1e-11, max_iter=200000)
    assert np.max(np.abs(x.cpu().numpy() - exact.x)) <= 1e-4


def test_dykstra_safeguard(mv):
    n, T = 900, 3500
    L, mu, Lq, mu_o, Rt = problem(mv, n, T, seed=59, pct=80)
    r0 = power_start(n)
    x, info = mv.npga_solve(L, mu, Rt, T, eps=1e-6, power_start=gpu(r0), proj_budget=1)
    assert info["dykstra"] >= 1
    assert info["converged"] == 1 and info["kkt"] <= 1e-6
    lam = power_norm2(Lq, r0, 50)
    exact = npga(Lq, 0.0, mu_o, Rt, initial_point(mu_o, Rt), step_size(lam, 0.0), eps=1e-11, max_iter=200000)
    assert np.max(np.abs(x.cpu().numpy() - exact.x)) <= 1e-4
    _, info0 = mv.npga_solve(L, mu, Rt, T, eps=1e-6, power_start=gpu(r0), proj_budget=1, dykstra_iters=0,
                             max_iter=200)
    assert info0["dykstra"] == 0 and info0["proj_failures"] >= 1


def test_variant_options_rejected(mv):
    n, T = 64, 300
    L, mu, _, _, Rt = problem(mv, n, T, seed=3)
    with pytest.raises(mv.MvError):
        mv.npga_solve(L, mu, Rt, T, momentum=1)              # gamma = 0 and no m_f
    with pytest.raises(mv.MvError):
        mv.npga_solve(L, mu, Rt, T, backtrack=1, bt_rho=1.5)
    with pytest.raises(mv.MvError):
        mv.npga_solve(L, mu, Rt, T, proj_budget=0)
