"""GPU parity of the Lanczos step-size estimate (mv_solve_opts.lanczos = 1).

lambda_hat is the top eigenvalue of the tridiagonal matrix of k Lanczos
steps on L L^T (the largest-singular-value option of the Sec. 3.1 fixed
step).  Expected values come from ``oracle.npga.lanczos_norm2`` on the FP64
copy of the stored factor; the products run in FP32, so lambda_hat agrees to
1e-5 relative (the tolerance of the power-method tests).  Solves that use
the estimate must reach the oracle's optimum like the power-method solves:
x within 1e-4 in the infinity norm, objective within 1e-5 relative.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import CFG_FULL, CFG_SMALL, factor_returns, power_start
from oracle.center import center_factor
from oracle.npga import (initial_point, kkt_residual, lanczos_norm2, lanczos_norm2_sigma, npga, objective,
                         power_norm2, sigma_from_factor, step_size)

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


def panel(n, T, seed, base=CFG_FULL):
    return factor_returns(base.scaled(n, T, seed=seed), np.float32)


def dequant(L, rs, n, T, dt, layout):
    """FP64 copy of the stored n x T factor (either layout)."""
    Lc = (L if layout == "nt" else L.t())[:n, :T]
    if dt == "f32":
        return Lc.double().cpu().numpy()
    if dt == "bf16":
        return Lc.float().double().cpu().numpy()
    q = Lc.cpu().view(torch.float8_e4m3fn).float().double().numpy()
    return q * rs.double().cpu().numpy()[:, None]


def lam_only(mv, L, mu, Rt, T, **kw):
    """lambda_hat and alpha of a solve that stops after its first KKT test."""
    _, info = mv.npga_solve(L, mu, Rt, T, eps=0.0, max_iter=0, **kw)
    return info


@pytest.mark.parametrize("layout", ["nt", "tn"])
@pytest.mark.parametrize("dt", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("shape", [(200, 1000), (777, 3001), (1536, 6000)])
def test_lanczos_lambda_parity(mv, layout, dt, shape):
    n, T = shape
    R32 = panel(n, T, seed=n + 3)
    L, rs, mu, _ = mv.center_factor(gpu(R32), dt, layout=layout)
    Lq = dequant(L, rs, n, T, dt, layout)
    r0 = power_start(n)
    Rt = float(np.percentile(mu.cpu().numpy(), 60))
    for k in (1, 2, 7, 25):
        info = lam_only(mv, L, mu, Rt, T, dtype=dt, row_scale=rs, layout=layout, power_start=gpu(r0),
                        lanczos=1, power_iters=k)
        assert info["lambda_hat"] == pytest.approx(lanczos_norm2(Lq, r0, k), rel=1e-5), k
        assert info["alpha"] == pytest.approx(step_size(info["lambda_hat"], 0.0), rel=1e-12)
    # never below the power method's estimate after k - 1 steps
    p24 = lam_only(mv, L, mu, Rt, T, dtype=dt, row_scale=rs, layout=layout, power_start=gpu(r0), power_iters=24)
    assert info["lambda_hat"] >= p24["lambda_hat"] * (1 - 1e-5)


@pytest.mark.parametrize("two_pass", [0, 1])
def test_lanczos_lambda_two_pass_and_sigma(mv, two_pass):
    n, T = 640, 2500
    R32 = panel(n, T, seed=11)
    L, rs, mu, _ = mv.center_factor(gpu(R32), "f32")
    L_o = dequant(L, rs, n, T, "f32", "nt")
    r0 = power_start(n)
    Rt = float(np.percentile(mu.cpu().numpy(), 60))
    info = lam_only(mv, L, mu, Rt, T, power_start=gpu(r0), lanczos=1, power_iters=20, two_pass=two_pass)
    assert info["lambda_hat"] == pytest.approx(lanczos_norm2(L_o, r0, 20), rel=1e-5)
    if two_pass == 0:
        S = sigma_from_factor(L_o).astype(np.float32)
        S_t = gpu(S)
        info_s = lam_only(mv, S_t, mu, Rt, n, layout="sigma", power_start=gpu(r0), lanczos=1, power_iters=20)
        assert info_s["lambda_hat"] == pytest.approx(lanczos_norm2_sigma(S.astype(np.float64), r0, 20), rel=1e-5)


def test_lanczos_degenerate_starts(mv):
    # A = diag(9, 4, 0, 0, 0): the Krylov space from 1 is 3-dimensional, the
    # estimate is 9 whatever the further steps do with the FP32 residual.
    n, T = 5, 2
    L = torch.zeros(n, 4, dtype=torch.float32, device=DEV)      # rows padded to 16 bytes
    L[0, 0], L[1, 1] = 3.0, 2.0
    mu = gpu(np.linspace(0.0, 1e-3, n))
    info = lam_only(mv, L, mu, 0.0, T, power_start=gpu(np.ones(n)), lanczos=1, power_iters=25)
    assert info["lambda_hat"] == pytest.approx(9.0, rel=1e-6)
    # a zero start vector gives no direction: lambda_hat = 0 (alpha falls back to 1)
    info0 = lam_only(mv, L, mu, 0.0, T, power_start=gpu(np.zeros(n)), lanczos=1, power_iters=25)
    assert info0["lambda_hat"] == 0.0 and info0["alpha"] == 1.0
    # one step: the Rayleigh quotient of the start vector
    info1 = lam_only(mv, L, mu, 0.0, T, power_start=gpu(np.ones(n)), lanczos=1, power_iters=1)
    assert info1["lambda_hat"] == pytest.approx(13.0 / 5.0, rel=1e-7)


def test_lanczos_option_checks(mv):
    n, T = 64, 256
    R32 = panel(n, T, seed=2)
    L, rs, mu, _ = mv.center_factor(gpu(R32), "f32")
    Rt = float(np.percentile(mu.cpu().numpy(), 60))
    for bad in (dict(lanczos=1, power_iters=0), dict(lanczos=1, power_iters=513), dict(lanczos=2)):
        with pytest.raises(mv.MvError):
            mv.npga_solve(L, mu, Rt, T, **bad)
    # with a given step the estimate is skipped, as for the power method
    x, info = mv.npga_solve(L, mu, Rt, T, alpha=0.5, lanczos=1, power_iters=0, max_iter=3, eps=0.0)
    assert info["lambda_hat"] == 0.0 and info["alpha"] == 0.5
    # the adjoint keeps the power method
    y = torch.ones(n, dtype=torch.float64, device=DEV)
    with pytest.raises(mv.MvError):
        mv.npga_backward(L, mu, Rt, T, y, 10, lanczos=1, power_iters=25)


@pytest.mark.parametrize("dt", ["bf16", "fp8"])
def test_lanczos_frontier(mv, dt):
    """The frontier's shared step from 25 Lanczos steps on the stored factor,
    and every target at the FP64 optimum of its own problem."""
    n, T = 300, 1500
    R32 = panel(n, T, seed=21)
    Lq_d, rs, mu, _ = mv.center_factor(gpu(R32), dt)
    Lq = dequant(Lq_d, rs, n, T, dt, "nt")
    mu_o = mu.cpu().numpy()
    r0 = power_start(n)
    targets = np.linspace(np.percentile(mu_o, 10), np.percentile(mu_o, 90), 8)
    fs = mv.FrontierSolver(Lq_d, mu, targets, T, eps=1e-7, dtype=dt, row_scale=rs, power_start=gpu(r0), lanczos=1,
                           power_iters=25)
    X, infos = fs.solve()
    lam_o = lanczos_norm2(Lq, r0, 25)
    for b, inf in enumerate(infos):
        assert inf["converged"] == 1
        assert inf["lambda_hat"] == pytest.approx(lam_o, rel=1e-5)
        ref = npga(Lq, 0.0, mu_o, float(targets[b]), initial_point(mu_o, float(targets[b])), step_size(lam_o, 0.0),
                   eps=1e-11, max_iter=200000)
        assert np.max(np.abs(X[b].cpu().numpy() - ref.x)) <= 1e-4


@pytest.mark.parametrize("layout", ["nt", "tn"])
@pytest.mark.parametrize("case", [(200, 1000, 0.0, "ge", 60), (900, 4000, 2e-5, "eq", 40)])
def test_lanczos_solve_parity(mv, layout, case):
    """Solve with the 25-step Lanczos step against the oracle's NPGA with the
    oracle's own 25-step estimate, and both against the FP64 optimum."""
    n, T, gamma, mode, pct = case
    R32 = panel(n, T, seed=n + 7, base=CFG_SMALL if n == 200 else CFG_FULL)
    L, rs, mu, _ = mv.center_factor(gpu(R32), "f32", layout=layout)
    mu_o, L_o, _ = center_factor(R32.astype(np.float64))
    Rt = float(np.percentile(mu_o, pct))
    r0 = power_start(n)
    x, info = mv.npga_solve(L, mu, Rt, T, gamma=gamma, mode=mode, layout=layout, power_start=gpu(r0), eps=1e-6,
                            lanczos=1, power_iters=25)
    assert info["converged"] == 1 and info["status"] == 0 and info["kkt"] <= 1e-6
    lam_o = lanczos_norm2(L_o, r0, 25)
    assert info["lambda_hat"] == pytest.approx(lam_o, rel=1e-5)
    x = x.cpu().numpy()
    ref = npga(L_o, gamma, mu_o, Rt, initial_point(mu_o, Rt, mode), step_size(lam_o, gamma), eps=1e-11,
               max_iter=200000, mode=mode)
    assert ref.converged
    assert np.max(np.abs(x - ref.x)) <= 1e-4
    f = objective(L_o, gamma, x)
    assert (f - ref.f) / ref.f <= 1e-5
    assert kkt_residual(L_o, gamma, mu_o, Rt, x, info["alpha"], mode) <= 1.05e-6
    # the same iterations as the oracle's loop on the same step (FP32 products)
    o6 = npga(L_o, gamma, mu_o, Rt, initial_point(mu_o, Rt, mode), step_size(lam_o, gamma), eps=1e-6,
              max_iter=200000, mode=mode)
    assert abs(info["iterations"] - o6.iters) <= 5


def test_lanczos_full_shape_sample(mv):
    """The 5440 x 48374 FP32 workload, stored transposed: the 25-step Lanczos
    estimate against the oracle's on the same stored factor, and above the
    50-step power estimate."""
    n, T = CFG_FULL.n, CFG_FULL.T
    R32 = factor_returns(CFG_FULL, np.float32)
    L, rs, mu, _ = mv.center_factor(gpu(R32), "f32", layout="tn")
    del R32
    L_o = dequant(L, rs, n, T, "f32", "tn")
    r0 = power_start(n)
    Rt = float(np.percentile(mu.cpu().numpy(), 60))
    info = lam_only(mv, L, mu, Rt, T, layout="tn", power_start=gpu(r0), lanczos=1, power_iters=25)
    lam_o = lanczos_norm2(L_o, r0, 25)
    assert info["lambda_hat"] == pytest.approx(lam_o, rel=1e-5)
    p50 = lam_only(mv, L, mu, Rt, T, layout="tn", power_start=gpu(r0), power_iters=50)
    assert info["lambda_hat"] > p50["lambda_hat"]


@pytest.mark.parametrize("lanczos", [0, 1])
def test_fp8_transposed_two_pass_estimates(mv, lanczos):
    """FP8 factor stored transposed, products as two passes: the FP32 copy of
    g that the power and Lanczos steps read carries the asset scales, so both
    estimates match the oracle's on the dequantised factor."""
    n, T = 900, 4000
    R32 = panel(n, T, seed=31)
    Lt, rs, mu, _ = mv.center_factor(gpu(R32), "fp8", layout="tn")
    Lq = dequant(Lt, rs, n, T, "fp8", "tn")
    r0 = power_start(n)
    Rt = float(np.percentile(mu.cpu().numpy(), 60))
    k = 25 if lanczos else 50
    info = lam_only(mv, Lt, mu, Rt, T, dtype="fp8", row_scale=rs, layout="tn", power_start=gpu(r0), two_pass=1,
                    lanczos=lanczos, power_iters=k)
    ref = lanczos_norm2(Lq, r0, k) if lanczos else power_norm2(Lq, r0, k)
    assert info["lambda_hat"] == pytest.approx(ref, rel=1e-5)
