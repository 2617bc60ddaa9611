"""GPU parity of the batched efficient-frontier solve (one BF16 factor, many
targets; skinny tcgen05 GEMMs) against the FP64 oracle on the same BF16
matrix.  Besides per-target parity, the frontier must be monotone: with the
return row active, the minimum variance cannot decrease as the target rises."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import CFG_FULL, CFG_SMALL, factor_returns, power_start
from oracle.center import center_factor
from oracle.npga import initial_point, npga, objective, power_norm2, step_size

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02917_gb300 import mv as m
    m.lib()
    return m


def oracle_opt(L64, mu, Rt):
    lam = power_norm2(L64, power_start(L64.shape[0]), 300)
    return npga(L64, 0.0, mu, Rt, initial_point(mu, Rt), step_size(lam, 0.0), eps=1e-11, max_iter=200000)


@pytest.mark.parametrize("model,nt", [(CFG_SMALL, 64), (CFG_FULL.scaled(700, 3001, seed=61), 5)])
def test_frontier_parity(mv, model, nt):
    R = factor_returns(model, np.float32)
    Lb, _, mu, _ = mv.center_factor(torch.from_numpy(R).cuda(), "bf16")
    mu_o = center_factor(R.astype(np.float64))[0]
    targets = np.linspace(np.percentile(mu_o, 10), np.percentile(mu_o, 90), nt)
    fs = mv.FrontierSolver(Lb, mu, targets, model.T, eps=1e-7)
    X, infos = fs.solve()
    X = X.cpu().numpy()
    assert all(i["converged"] == 1 for i in infos)
    Lq = Lb[:, :model.T].float().double().cpu().numpy()      # the BF16 model the GPU holds
    f = np.array([objective(Lq, 0.0, X[b]) for b in range(nt)])
    for b in range(nt):
        assert X[b].min() >= 0 and abs(X[b].sum() - 1) < 1e-12 and mu_o @ X[b] >= targets[b] - 1e-15
        assert infos[b]["objective"] == pytest.approx(f[b], rel=1e-4)
    check = range(nt) if nt <= 8 else range(0, nt, 9)
    for b in check:
        ref = oracle_opt(Lq, mu_o, targets[b])
        assert np.max(np.abs(X[b] - ref.x)) <= 1e-4
        assert (f[b] - ref.f) / ref.f <= 1e-5
    # monotone frontier where the return row binds
    active = [b for b in range(nt) if abs(mu_o @ X[b] - targets[b]) < 1e-12]
    fa = f[active]
    assert np.all(np.diff(fa) >= -1e-12 * fa.max())


@pytest.mark.parametrize("model,nt", [(CFG_SMALL, 64), (CFG_FULL.scaled(700, 3001, seed=62), 7)])
def test_frontier_fp8_parity(mv, model, nt):
    """FP8 e4m3 factor with row scales: FP8 tiles expanded to BF16 in shared
    memory before the tcgen05 MMA; parity against the oracle on the FP8 model."""
    R = factor_returns(model, np.float32)
    Lq, rs, mu, _ = mv.center_factor(torch.from_numpy(R).cuda(), "fp8")
    mu_o = center_factor(R.astype(np.float64))[0]
    targets = np.linspace(np.percentile(mu_o, 10), np.percentile(mu_o, 90), nt)
    fs = mv.FrontierSolver(Lq, mu, targets, model.T, eps=1e-7, dtype="fp8", row_scale=rs)
    X, infos = fs.solve()
    X = X.cpu().numpy()
    assert all(i["converged"] == 1 for i in infos)
    q = Lq[:, :model.T].cpu().view(torch.float8_e4m3fn).float().double().numpy()
    L8 = q * rs.double().cpu().numpy()[:, None]                 # the FP8 model the GPU holds
    f = np.array([objective(L8, 0.0, X[b]) for b in range(nt)])
    for b in range(nt):
        assert X[b].min() >= 0 and abs(X[b].sum() - 1) < 1e-12 and mu_o @ X[b] >= targets[b] - 1e-15
        assert infos[b]["objective"] == pytest.approx(f[b], rel=1e-4)
    for b in (range(nt) if nt <= 8 else range(0, nt, 9)):
        ref = oracle_opt(L8, mu_o, targets[b])
        assert np.max(np.abs(X[b] - ref.x)) <= 1e-4
        assert (f[b] - ref.f) / ref.f <= 1e-5


@pytest.mark.slow
@pytest.mark.parametrize("dt", ["bf16", "fp8", "bf16+f32"])
def test_frontier_full_shape_against_oracle(mv, dt):
    """The 64-target frontier at 5440 x 48374, launched as the benchmark
    launches it (targets evenly spaced between the 10th and 90th percentiles
    of mu, KKT 1e-6).  Three targets -- the 10th percentile, the middle of the
    grid and the 90th percentile -- are checked against the oracle's optimum
    on the same low-precision matrix: Algorithm 1 in FP64 on Sigma = L L^T
    from Pi_F(1/n 1) to a KKT residual of 1e-10.  Tolerances as for the
    single solves: x within 1e-4 (infinity norm), objective within 1e-5
    relative, and f(x) - f* within the Frank--Wolfe gap at x.  "bf16+f32" is
    the BF16 frontier refined on the FP32 factor, checked against the oracle
    on the FP32 model (the oracle's own L rounded to FP32)."""
    from oracle.npga import fw_gap, npga_sigma, objective_sigma, power_norm2_sigma, sigma_from_factor
    m = CFG_FULL
    R = factor_returns(m, np.float32)
    refine = dt == "bf16+f32"
    Rd = torch.from_numpy(R).cuda()
    Lq_d, rs, mu, _ = mv.center_factor(Rd, "bf16" if refine else dt)
    L32 = mv.center_factor(Rd, "f32")[0] if refine else None
    del Rd
    mu_o, L_o, _ = center_factor(R.astype(np.float64))
    del R
    targets = np.linspace(np.percentile(mu_o, 10), np.percentile(mu_o, 90), 64)
    fs = mv.FrontierSolver(Lq_d, mu, targets, m.T, eps=1e-6, dtype="bf16" if refine else dt, row_scale=rs,
                           L_f32=L32, eps_lo=1e-5)
    X, infos = fs.solve()
    X = X.cpu().numpy()
    assert all(i["converged"] == 1 for i in infos)
    if refine:
        Lq = L_o.astype(np.float32).astype(np.float64)
    elif dt == "bf16":
        Lq = Lq_d[:, :m.T].float().double().cpu().numpy()
    else:
        q = Lq_d[:, :m.T].cpu().view(torch.float8_e4m3fn).float().double().numpy()
        Lq = q * rs.double().cpu().numpy()[:, None]
    del fs, Lq_d, L_o, L32
    Sig = sigma_from_factor(Lq)
    alpha = 1.0 / (2.0 * power_norm2_sigma(Sig, power_start(m.n), 100) * (1 + 1e-3))
    for b in (0, 32, 63):
        ref = npga_sigma(Sig, 0.0, mu_o, targets[b], initial_point(mu_o, targets[b]), alpha, eps=1e-10,
                         max_iter=50000)
        assert ref.converged
        x = X[b]
        assert x.min() >= 0 and abs(x.sum() - 1) < 1e-12 and mu_o @ x >= targets[b] - 1e-15
        f = objective_sigma(Sig, 0.0, x)
        assert np.max(np.abs(x - ref.x)) <= 1e-4
        assert (f - ref.f) / ref.f <= 1e-5
        assert -1e-14 * ref.f <= f - ref.f <= fw_gap(Lq, 0.0, mu_o, targets[b], x) + 1e-12 * ref.f
        assert infos[b]["objective"] == pytest.approx(f, rel=1e-4)


@pytest.mark.parametrize("model,nt,dt", [(CFG_SMALL, 64, "bf16"), (CFG_FULL.scaled(700, 3001, seed=63), 7, "fp8")])
def test_frontier_refined_reaches_fp32_optimum(mv, model, nt, dt):
    """Low-precision frontier to KKT 1e-5, then every target refined on the
    FP32 factor (BF16 hi + lo pair, 2^-18 per entry) to 1e-6: parity with the
    oracle on the FP32 model (the oracle's own centering rounded to FP32, which
    is the GPU's FP32 factor bit for bit)."""
    from oracle.npga import kkt_residual
    R = factor_returns(model, np.float32)
    Rd = torch.from_numpy(R).cuda()
    Lq, rs, mu, _ = mv.center_factor(Rd, dt)
    L32, _, _, _ = mv.center_factor(Rd, "f32")
    mu_o, L_o, _ = center_factor(R.astype(np.float64))
    L_o = L_o.astype(np.float32).astype(np.float64)
    targets = np.linspace(np.percentile(mu_o, 10), np.percentile(mu_o, 90), nt)
    fs = mv.FrontierSolver(Lq, mu, targets, model.T, dtype=dt, row_scale=rs, L_f32=L32, eps_lo=1e-5, eps=1e-6)
    X, infos = fs.solve()
    X = X.cpu().numpy()
    assert all(i["converged"] == 1 and i["kkt"] <= 1e-6 for i in infos)
    assert all(0 <= i["refine_iterations"] <= i["iterations"] for i in infos)
    for b in (range(nt) if nt <= 8 else range(0, nt, 9)):
        ref = oracle_opt(L_o, mu_o, targets[b])
        x = X[b]
        assert x.min() >= 0 and abs(x.sum() - 1) < 1e-12 and mu_o @ x >= targets[b] - 1e-15
        assert np.max(np.abs(x - ref.x)) <= 1e-4
        f = objective(L_o, 0.0, x)
        assert (f - ref.f) / ref.f <= 1e-5
        assert infos[b]["objective"] == pytest.approx(f, rel=1e-4)
        assert kkt_residual(L_o, 0.0, mu_o, targets[b], x, infos[b]["alpha"]) <= 1.5e-6
