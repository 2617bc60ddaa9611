"""GPU parity: libmv (through the C ABI) against the FP64 oracle.

Inputs come from ``synth`` only; expected values come from ``oracle`` only.
Tolerances: centering exact up to the FP32 rounding of L; projection FP64
(1e-12 absolute, active set identical off the degenerate set); FP32 products
1e-5 relative; solver x within 1e-4 in the infinity norm and objective within
1e-5 relative of the oracle's optimum.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import CFG_FULL, CFG_SMALL, factor_returns, power_start
from oracle.center import center_factor
from oracle.projection import PROJ_OK, active_set, project_F
from oracle.npga import (fw_gap, gradient, initial_point, kkt_residual, npga, npga_sigma, objective,
                         objective_sigma, power_norm2, power_norm2_sigma, sigma_from_factor, step_size)

pytestmark = pytest.mark.gpu

GOLD_PATH = __file__.replace("test_gpu_parity.py", "golden/hand_cases.json")


@pytest.fixture(scope="module")
def mv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02917_gb300 import mv as m
    m.lib()
    return m


DEV = "cuda:0"


def gpu(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


def panel(n, T, seed, base=CFG_SMALL):
    R32 = factor_returns(base.scaled(n, T, seed=seed), np.float32)
    return R32, R32.astype(np.float64)


def dequant(mv, L, rs, T, dt):
    if dt == "f32":
        return L[:, :T].double().cpu().numpy()
    if dt == "bf16":
        return L[:, :T].float().double().cpu().numpy()
    q = L[:, :T].cpu().view(torch.float8_e4m3fn).float().double().numpy()
    return q * rs.double().cpu().numpy()[:, None]


# ------------------------------------------------------------------ centering
@pytest.mark.parametrize("dt", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("shape", [(37, 1001), (5, 2), (1, 3), (300, 4099)])
def test_center_parity(mv, dt, shape):
    n, T = shape
    R32, R64 = panel(n, T, seed=3)
    L, rs, mu, tr = mv.center_factor(gpu(R32), dt)
    mu_o, L_o, tr_o = center_factor(R64)
    np.testing.assert_allclose(mu.cpu().numpy(), mu_o, rtol=1e-14, atol=1e-18)
    assert float(tr.cpu()) == pytest.approx(tr_o, rel=1e-12)
    Lg = dequant(mv, L, rs, T, dt)
    if dt == "f32":
        # exactly the FP32 rounding of the FP64 centered value
        np.testing.assert_array_equal(Lg, L_o.astype(np.float32).astype(np.float64))
    elif dt == "bf16":
        np.testing.assert_allclose(Lg, L_o, rtol=2.0 ** -8, atol=1e-30)
    else:
        # e4m3 with a per-row scale: relative step 2^-3, subnormal floor 2^-9 * scale
        scale = rs.double().cpu().numpy()[:, None]
        assert np.all(np.abs(Lg - L_o) <= 2.0 ** -4 * np.abs(L_o) + 2.0 ** -10 * scale + 1e-30)
        np.testing.assert_allclose(scale[:, 0], np.abs(L_o).max(axis=1) / 448.0, rtol=1e-6)
    pad = L[:, T:]
    assert pad.numel() == 0 or int((pad.float() != 0).sum()) == 0


# ------------------------------------------------------------------ projection
def test_project_hand_cases(mv):
    import json
    gold = json.load(open(GOLD_PATH))
    for c in gold["projection_F"]:
        x, info = mv.project(gpu(np.array(c["v"])), gpu(np.array(c["mu"])), c["R"], c["mode"])
        assert info["status"] == 0
        np.testing.assert_allclose(x.cpu().numpy(), c["x"], atol=1e-13)
        if c["nu"] is not None:
            assert info["nu"] == pytest.approx(c["nu"], rel=1e-10)
            assert info["tau"] == pytest.approx(c["tau"], rel=1e-10, abs=1e-12)


@pytest.mark.parametrize("mode", ["ge", "eq"])
@pytest.mark.parametrize("n", [1, 2, 3, 7, 64, 513, 1025, 2000, 5440, 13001, 32768])
def test_project_random_parity(mv, n, mode):
    rng = np.random.default_rng(1000 + n + (7 if mode == "eq" else 0))
    batch = 6
    mu = rng.uniform(-2e-4, 6e-4, n)
    V = rng.standard_normal((batch, n)) * 3e-3 + 1.0 / n
    Rt = np.array([np.percentile(mu, q) for q in np.linspace(5, 99, batch)])
    if n == 1:
        Rt[:] = mu[0]
    x, infos = mv.project(gpu(V), gpu(mu), gpu(Rt), mode)
    x = x.cpu().numpy()
    for b in range(batch):
        p = project_F(V[b], mu, Rt[b], mode)
        assert p.status == PROJ_OK
        assert infos[b]["status"] == 0, infos[b]
        np.testing.assert_allclose(x[b], p.x, rtol=0, atol=1e-12)
        act, deg = active_set(V[b], mu, p.nu, p.tau)
        assert np.array_equal((x[b] > 0)[~deg], act[~deg])
        assert infos[b]["support"] == int((x[b] > 0).sum())
        assert abs(x[b].sum() - 1.0) < 1e-12 and x[b].min() >= 0.0


def test_project_infeasible_and_edges(mv):
    mu = np.array([0.01, 0.02, 0.03])
    v = np.array([[0.2, 0.3, 0.5], [0.2, 0.3, 0.5], [0.9, 0.05, 0.05]])
    Rt = np.array([0.031, 0.03, 0.0])
    x, infos = mv.project(gpu(v), gpu(mu), gpu(Rt), "ge")
    x = x.cpu().numpy()
    assert infos[0]["status"] == mv.MV_ERR_INFEASIBLE and np.all(np.isnan(x[0]))
    np.testing.assert_allclose(x[1], [0.0, 0.0, 1.0], atol=1e-14)        # R = max mu
    np.testing.assert_allclose(x[2], project_F(v[2], mu, 0.0).x, atol=1e-14)
    _, infos = mv.project(gpu(v[:1]), gpu(mu), gpu(np.array([0.005])), "eq")
    assert infos[0]["status"] == mv.MV_ERR_INFEASIBLE                     # R < min mu
    # NaN in the point: reported, not hung
    vv = v[:1].copy()
    vv[0, 1] = np.nan
    _, infos = mv.project(gpu(vv), gpu(mu), gpu(np.array([0.025])), "ge")
    assert infos[0]["status"] in (mv.MV_ERR_NUMERIC, mv.MV_ERR_NOT_CONVERGED)


# ------------------------------------------------------------------ products
@pytest.mark.parametrize("dt", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("shape", [(200, 1000), (333, 4999), (1, 17), (2100, 9001)])
def test_gradient_parity(mv, dt, shape):
    n, T = shape
    R32, _ = panel(n, T, seed=5)
    L, rs, mu, _ = mv.center_factor(gpu(R32), dt)
    Lq = dequant(mv, L, rs, T, dt)            # the matrix the GPU actually holds
    y = np.random.default_rng(2).dirichlet(np.ones(n))
    gamma = 3e-5
    z, g = mv.gradient(L, gpu(y), T, gamma, dt, rs)
    z_o = Lq.T @ y
    g_o = gradient(Lq, gamma, y)
    # FP32 accumulation over n (z) and T (g) terms
    assert np.max(np.abs(z.cpu().numpy() - z_o)) <= 2e-5 * np.max(np.abs(z_o)) + 1e-30
    assert np.max(np.abs(g.cpu().numpy() - g_o)) <= 2e-5 * np.max(np.abs(g_o)) + 1e-30


# Fused single pass g = L L^T y (one HBM pass; applies for n >= 1024, T >= 4096).
# Shapes: exact multiples, ragged T (partial last column block), ragged n (the
# last CTA of a cluster holds rows past n), and the largest n with 3 stages.
@pytest.mark.parametrize("dt", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("shape", [(1024, 4096), (1030, 4099), (2100, 9001), (5440, 6007)])
def test_gradient_fused_parity(mv, dt, shape):
    n, T = shape
    R32, _ = panel(n, T, seed=7)
    L, rs, mu, _ = mv.center_factor(gpu(R32), dt)
    Lq = dequant(mv, L, rs, T, dt)
    y = np.random.default_rng(3).dirichlet(np.ones(n))
    gamma = 1e-5
    zf, gf = mv.gradient(L, gpu(y), T, gamma, dt, rs, with_z=False)
    assert zf is None
    # with z requested the same single pass also writes the slices of z = L^T y it forms
    z2, g2 = mv.gradient(L, gpu(y), T, gamma, dt, rs, with_z=True)
    g_o = gradient(Lq, gamma, y)
    z_o = Lq.T @ y
    gf = gf.cpu().numpy()
    assert np.max(np.abs(gf - g_o)) <= 2e-5 * np.max(np.abs(g_o))
    assert np.array_equal(gf, g2.cpu().numpy())
    assert np.max(np.abs(z2.cpu().numpy() - z_o)) <= 2e-5 * np.max(np.abs(z_o))
    # deterministic: the same bits on a second call
    _, gf2 = mv.gradient(L, gpu(y), T, gamma, dt, rs, with_z=False)
    assert np.array_equal(gf, gf2.cpu().numpy())


@pytest.mark.parametrize("shape", [(6400, 4100), (8200, 4096), (16000, 4096)])
def test_gradient_fused_larger_clusters(mv, shape):
    """n past a 2-CTA cluster's row capacity: clusters of 4 and 8 CTAs."""
    n, T = shape
    R32, _ = panel(n, T, seed=8)
    L, rs, mu, _ = mv.center_factor(gpu(R32), "f32")
    y = np.random.default_rng(4).dirichlet(np.ones(n))
    _, gf = mv.gradient(L, gpu(y), T, 0.0, "f32", rs, with_z=False)
    g_o = gradient(L[:, :T].double().cpu().numpy(), 0.0, y)
    assert np.max(np.abs(gf.cpu().numpy() - g_o)) <= 2e-5 * np.max(np.abs(g_o))


@pytest.mark.parametrize("dt", ["f32", "bf16"])
@pytest.mark.parametrize("case", [(1500, 6000, 0.0, "ge", 60), (1100, 4500, 2e-5, "eq", 40)])
def test_npga_fused_parity(mv, dt, case):
    n, T, gamma, mode, pct = case
    R32, R64 = panel(n, T, seed=n + 1, base=CFG_FULL)
    L, rs, mu, _ = mv.center_factor(gpu(R32), dt)
    Lq = dequant(mv, L, rs, T, dt)
    mu_o = mu.cpu().numpy()
    Rt = float(np.percentile(mu_o, pct))
    r0 = power_start(n)
    x, info = mv.npga_solve(L, mu, Rt, T, gamma=gamma, dtype=dt, row_scale=rs, mode=mode, eps=1e-6,
                            power_start=gpu(r0))
    assert info["fused"] == 1
    assert info["converged"] == 1 and info["status"] == 0 and info["kkt"] <= 1e-6
    assert info["lambda_hat"] == pytest.approx(power_norm2(Lq, r0, 50), rel=1e-5)
    x = x.cpu().numpy()
    ref = oracle_solution(Lq, mu_o, Rt, gamma, mode)
    assert np.max(np.abs(x - ref.x)) <= 1e-4
    f = objective(Lq, gamma, x)
    assert (f - ref.f) / ref.f <= 1e-5
    assert info["objective"] == pytest.approx(f, rel=1e-5)
    assert kkt_residual(Lq, gamma, mu_o, Rt, x, info["alpha"], mode) <= 1.05e-6
    # the two-pass loop reaches the same point
    x2, info2 = mv.npga_solve(L, mu, Rt, T, gamma=gamma, dtype=dt, row_scale=rs, mode=mode, eps=1e-6,
                              power_start=gpu(r0), two_pass=1)
    assert info2["fused"] == 0 and info2["converged"] == 1
    assert np.max(np.abs(x2.cpu().numpy() - x)) <= 1e-5


# ------------------------------------------------------------------ NPGA
def oracle_solution(L64, mu, Rt, gamma=0.0, mode="ge"):
    lam = power_norm2(L64, power_start(L64.shape[0]), 200)
    x0 = initial_point(mu, Rt, mode)
    return npga(L64, gamma, mu, Rt, x0, step_size(lam, gamma), eps=1e-11, max_iter=200000, mode=mode)


def test_npga_small_config_2000_iterations(mv):
    """200 assets x 1000 periods, 2000 iterations, FP32 products vs FP64 oracle."""
    R32, R64 = panel(CFG_SMALL.n, CFG_SMALL.T, seed=CFG_SMALL.seed)
    L, _, mu, _ = mv.center_factor(gpu(R32), "f32")
    mu_o, L_o, _ = center_factor(R64)
    Rt = float(np.percentile(mu_o, 60))
    r0 = power_start(CFG_SMALL.n)
    x, info = mv.npga_solve(L, mu, Rt, CFG_SMALL.T, power_start=gpu(r0), eps=0.0, max_iter=2000)
    x = x.cpu().numpy()
    assert info["iterations"] == 2000
    # same power estimate as the oracle's 50 steps from the same start
    assert info["lambda_hat"] == pytest.approx(power_norm2(L_o, r0, 50), rel=1e-5)
    ref = oracle_solution(L_o, mu_o, Rt)
    assert np.max(np.abs(x - ref.x)) <= 1e-4
    f = objective(L_o, 0.0, x)
    assert abs(f - ref.f) / ref.f <= 1e-5
    assert info["objective"] == pytest.approx(f, rel=1e-5)
    assert x.min() >= 0 and abs(x.sum() - 1) < 1e-12 and mu_o @ x >= Rt - 1e-15
    assert kkt_residual(L_o, 0.0, mu_o, Rt, x, info["alpha"]) <= 1e-6


@pytest.mark.parametrize("dt", ["f32"])
@pytest.mark.parametrize("case", [(700, 5003, 0.0, "ge", 60), (1024, 3000, 2e-5, "ge", 75),
                                  (400, 2500, 0.0, "eq", 30), (129, 777, 0.0, "ge", 97)])
def test_npga_to_kkt_parity(mv, dt, case):
    n, T, gamma, mode, pct = case
    R32, R64 = panel(n, T, seed=n, base=CFG_FULL)
    L, rs, mu, _ = mv.center_factor(gpu(R32), dt)
    mu_o, L_o, _ = center_factor(R64)
    Rt = float(np.percentile(mu_o, pct))
    x, info = mv.npga_solve(L, mu, Rt, T, gamma=gamma, dtype=dt, row_scale=rs, mode=mode, eps=1e-6)
    assert info["converged"] == 1 and info["status"] == 0 and info["kkt"] <= 1e-6
    assert info["iterations"] % 5 == 0
    x = x.cpu().numpy()
    ref = oracle_solution(L_o, mu_o, Rt, gamma, mode)
    assert np.max(np.abs(x - ref.x)) <= 1e-4
    f = objective(L_o, gamma, x)
    assert (f - ref.f) / ref.f <= 1e-5
    assert kkt_residual(L_o, gamma, mu_o, Rt, x, info["alpha"], mode) <= 1.05e-6


def test_npga_warm_start_alpha_override_and_budget(mv):
    n, T = 150, 900
    R32, R64 = panel(n, T, seed=8)
    L, _, mu, _ = mv.center_factor(gpu(R32), "f32")
    mu_o, L_o, _ = center_factor(R64)
    Rt = float(np.percentile(mu_o, 60))
    lam = power_norm2(L_o, power_start(n), 500)
    alpha = step_size(lam, 0.0, 0.0)
    # budget exhausted -> NOT_CONVERGED with the last iterate and its residual
    x, info = mv.npga_solve(L, mu, Rt, T, alpha=alpha, eps=1e-14, max_iter=12)
    assert info["status"] == mv.MV_ERR_NOT_CONVERGED and info["iterations"] == 12
    assert info["alpha"] == alpha and info["lambda_hat"] == 0.0
    xo = npga(L_o, 0.0, mu_o, Rt, initial_point(mu_o, Rt), alpha, eps=0.0, max_iter=12, kkt_every=0).x
    np.testing.assert_allclose(x.cpu().numpy(), xo, atol=1e-6)
    # warm start from that point converges to the same optimum as a cold start
    x2, info2 = mv.npga_solve(L, mu, Rt, T, alpha=alpha, eps=1e-8, x0=x.clone(), max_iter=20000)
    ref = oracle_solution(L_o, mu_o, Rt)
    assert info2["converged"] == 1
    assert np.max(np.abs(x2.cpu().numpy() - ref.x)) <= 1e-5


def test_npga_infeasible_target(mv):
    R32, R64 = panel(50, 300, seed=9)
    L, _, mu, _ = mv.center_factor(gpu(R32), "f32")
    Rt = float(mu.max().cpu()) + 1e-6
    with pytest.raises(mv.MvError) as e:
        mv.npga_solve(L, mu, Rt, 300)
    assert e.value.status == mv.MV_ERR_INFEASIBLE


@pytest.mark.parametrize("kkt_every,graph", [(1, 1), (5, 0), (7, 1)])
def test_npga_check_period_and_graph_modes(mv, kkt_every, graph):
    R32, R64 = panel(260, 1500, seed=12)
    L, _, mu, _ = mv.center_factor(gpu(R32), "f32")
    mu_o, L_o, _ = center_factor(R64)
    Rt = float(np.percentile(mu_o, 65))
    x, info = mv.npga_solve(L, mu, Rt, 1500, eps=1e-7, kkt_every=kkt_every, use_graph=graph)
    assert info["converged"] == 1 and info["iterations"] % kkt_every == 0
    ref = oracle_solution(L_o, mu_o, Rt)
    assert np.max(np.abs(x.cpu().numpy() - ref.x)) <= 1e-5


@pytest.mark.slow
def test_npga_full_size_against_oracle_optimum(mv):
    """The 5440 x 48374 FP32 workload (1.05 GB) launched as the benchmark
    launches it: L^T stored T x n, fused single pass, power start of seed 7,
    KKT residual 1e-6 tested every 5 iterations.

    The oracle centres the same panel in FP64 and rounds L to FP32 (the
    GPU's L is that rounding, bit for bit: test_center_parity), forms
    Sigma = L L^T in FP64 and runs Algorithm 1 on it from its own start
    x^0 = Pi_F(1/n 1) to a KKT residual of 1e-10, which gives x*.  The GPU's
    x must lie within 1e-4 of x* in the infinity norm with its objective
    within 1e-5 relative, and the Frank--Wolfe gap at x must bound
    f(x) - f* (Sec. 5.2's gap metric certified: the FW gap is an upper bound
    on the suboptimality of any feasible point of a convex problem)."""
    m = CFG_FULL
    R32 = factor_returns(m, np.float32)
    L, _, mu, _ = mv.center_factor(gpu(R32), "f32", layout="tn")
    mu_o, L_o, _ = center_factor(R32.astype(np.float64))
    del R32
    L_o = L_o.astype(np.float32).astype(np.float64)
    Rt = float(np.percentile(mu_o, 60))
    r0 = power_start(m.n)
    x, info = mv.npga_solve(L, mu, Rt, m.T, eps=1e-6, layout="tn", power_start=gpu(r0))
    assert info["converged"] == 1 and info["kkt"] <= 1e-6 and info["fused"] == 1
    x = x.cpu().numpy()
    del L
    assert x.min() >= 0 and abs(x.sum() - 1) < 1e-12 and mu_o @ x >= Rt - 1e-15
    assert kkt_residual(L_o, 0.0, mu_o, Rt, x, info["alpha"]) <= 1.05e-6
    Sig = sigma_from_factor(L_o)
    ref = npga_sigma(Sig, 0.0, mu_o, Rt, initial_point(mu_o, Rt), step_size(power_norm2_sigma(Sig, r0, 100), 0.0),
                     eps=1e-10, max_iter=50000)
    assert ref.converged
    f = objective_sigma(Sig, 0.0, x)
    assert np.max(np.abs(x - ref.x)) <= 1e-4
    assert (f - ref.f) / ref.f <= 1e-5
    assert info["objective"] == pytest.approx(f, rel=1e-5)
    gap = fw_gap(L_o, 0.0, mu_o, Rt, x)
    assert -1e-14 * ref.f <= f - ref.f <= gap + 1e-12 * ref.f


# ------------------------------------------------------------------ low precision
@pytest.mark.parametrize("dt", ["bf16", "fp8"])
def test_npga_low_precision_model_parity(mv, dt):
    """The solve on the BF16 / FP8 copy matches the oracle on that same (dequantized) matrix."""
    n, T = 700, 5003
    R32, R64 = panel(n, T, seed=31, base=CFG_FULL)
    L, rs, mu, _ = mv.center_factor(gpu(R32), dt)
    Lq = dequant(mv, L, rs, T, dt)
    mu_o = center_factor(R64)[0]
    Rt = float(np.percentile(mu_o, 60))
    x, info = mv.npga_solve(L, mu, Rt, T, dtype=dt, row_scale=rs, eps=1e-6)
    assert info["converged"] == 1
    x = x.cpu().numpy()
    ref = oracle_solution(Lq, mu_o, Rt)
    assert np.max(np.abs(x - ref.x)) <= 1e-4
    assert (objective(Lq, 0.0, x) - ref.f) / ref.f <= 1e-5


@pytest.mark.parametrize("dt", ["bf16", "fp8"])
def test_npga_refined_reaches_fp32_optimum(mv, dt):
    """Low-precision phase + FP32 refinement lands on the FP32 model's optimum."""
    n, T = 900, 6001
    R32, R64 = panel(n, T, seed=32, base=CFG_FULL)
    Rd = gpu(R32)
    L32, _, mu, _ = mv.center_factor(Rd, "f32")
    Llo, rs, _, _ = mv.center_factor(Rd, dt)
    mu_o, L_o, _ = center_factor(R64)
    Rt = float(np.percentile(mu_o, 60))
    s = mv.RefinedSolver(Llo, L32, mu, Rt, T, dtype=dt, row_scale=rs, eps_lo=1e-5, eps=1e-6)
    x, info = s.solve()
    assert info["converged"] == 1 and info["kkt"] <= 1e-6 and info["refine_iterations"] >= 0
    x = x.cpu().numpy()
    ref = oracle_solution(L_o, mu_o, Rt)
    assert np.max(np.abs(x - ref.x)) <= 1e-4
    assert (objective(L_o, 0.0, x) - ref.f) / ref.f <= 1e-5
    assert kkt_residual(L_o, 0.0, mu_o, Rt, x, info["alpha"]) <= 1.05e-6
