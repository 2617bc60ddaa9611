"""GPU parity of the transposed factor layout (MV_LAYOUT_TN: L^T stored T x n).

The centering writes the same values as the n x T layout, only transposed;
the products (two-pass and fused single pass) and the solve are checked
against the FP64 oracle on the matrix the GPU holds, with the tolerances of
test_gpu_parity (FP32 products 2e-5 of the largest entry; solver x within
1e-4, objective within 1e-5 relative).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import CFG_FULL, CFG_SMALL, factor_returns, power_start
from oracle.npga import gradient, initial_point, kkt_residual, npga, objective, power_norm2, step_size

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


def panel(n, T, seed, base=CFG_SMALL):
    return factor_returns(base.scaled(n, T, seed=seed), np.float32)


def held(mv, Lt, rs, n, dt):
    """The n x T matrix the GPU holds, from the T x ld transposed storage."""
    if dt == "f32":
        q = Lt[:, :n].double()
    elif dt == "bf16":
        q = Lt[:, :n].float().double()
    else:
        q = Lt[:, :n].cpu().view(torch.float8_e4m3fn).float().double()
    q = q.cpu().numpy().T
    if dt == "fp8":
        q = q * rs.double().cpu().numpy()[:, None]
    return q


@pytest.mark.parametrize("dt", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("shape", [(37, 1001), (300, 4099), (1030, 70)])
def test_center_tn_is_transpose(mv, dt, shape):
    n, T = shape
    R = gpu(panel(n, T, seed=11))
    L, rs, mu, tr = mv.center_factor(R, dt)
    Lt, rst, mut, trt = mv.center_factor(R, dt, layout="tn")
    assert Lt.shape[0] == T and Lt.shape[1] >= n
    assert torch.equal(mu, mut)
    # the trace is summed in a different (fixed) order per layout: FP64 rounding apart
    assert float(trt) == pytest.approx(float(tr), rel=1e-13)
    if dt == "fp8":
        assert torch.equal(rs, rst)
    a = L[:, :T].contiguous().view(torch.uint8 if dt == "fp8" else L.dtype).cpu()
    b = Lt[:, :n].t().contiguous().view(torch.uint8 if dt == "fp8" else Lt.dtype).cpu()
    assert torch.equal(a, b)
    assert torch.count_nonzero(Lt[:, n:].view(torch.uint8) if dt == "fp8" else Lt[:, n:]) == 0


@pytest.mark.parametrize("dt", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("shape", [(200, 1000), (1030, 4099), (2100, 9001), (5440, 6007), (7000, 4100)])
def test_gradient_tn_parity(mv, dt, shape):
    n, T = shape
    R = gpu(panel(n, T, seed=13))
    Lt, rs, mu, _ = mv.center_factor(R, dt, layout="tn")
    Lq = held(mv, Lt, rs, n, dt)
    y = np.random.default_rng(5).dirichlet(np.ones(n))
    gamma = 2e-5
    g_o = gradient(Lq, gamma, y)
    z2, g2 = mv.gradient(Lt, gpu(y), T, gamma, dt, rs, with_z=True, layout="tn")
    z_o = Lq.T @ y
    assert np.max(np.abs(z2.cpu().numpy() - z_o)) <= 2e-5 * np.max(np.abs(z_o))
    assert np.max(np.abs(g2.cpu().numpy() - g_o)) <= 2e-5 * np.max(np.abs(g_o))
    _, gf = mv.gradient(Lt, gpu(y), T, gamma, dt, rs, with_z=False, layout="tn")
    gf = gf.cpu().numpy()
    assert np.max(np.abs(gf - g_o)) <= 2e-5 * np.max(np.abs(g_o))
    _, gf2 = mv.gradient(Lt, gpu(y), T, gamma, dt, rs, with_z=False, layout="tn")
    assert np.array_equal(gf, gf2.cpu().numpy())          # deterministic


def oracle_solution(L64, mu, Rt, gamma=0.0, mode="ge"):
    lam = power_norm2(L64, power_start(L64.shape[0]), 200)
    x0 = initial_point(mu, Rt, mode)
    return npga(L64, gamma, mu, Rt, x0, step_size(lam, gamma), eps=1e-11, max_iter=200000, mode=mode)


@pytest.mark.parametrize("dt", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("case", [(1500, 6000, 0.0, "ge", 60), (1100, 4500, 2e-5, "eq", 40)])
def test_npga_tn_parity(mv, dt, case):
    n, T, gamma, mode, pct = case
    R = gpu(panel(n, T, seed=n + 3, base=CFG_FULL))
    Lt, rs, mu, _ = mv.center_factor(R, dt, layout="tn")
    Lq = held(mv, Lt, rs, n, dt)
    mu_o = mu.cpu().numpy()
    Rt = float(np.percentile(mu_o, pct))
    r0 = power_start(n)
    x, info = mv.npga_solve(Lt, mu, Rt, T, gamma=gamma, dtype=dt, row_scale=rs, mode=mode, eps=1e-6,
                            power_start=gpu(r0), layout="tn")
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
    x2, info2 = mv.npga_solve(Lt, mu, Rt, T, gamma=gamma, dtype=dt, row_scale=rs, mode=mode, eps=1e-6,
                              power_start=gpu(r0), layout="tn", two_pass=1)
    assert info2["fused"] == 0 and info2["converged"] == 1
    assert np.max(np.abs(x2.cpu().numpy() - x)) <= 1e-5


def test_refined_tn(mv):
    n, T = 1200, 5000
    R = gpu(panel(n, T, seed=21, base=CFG_FULL))
    Lb, _, mu, _ = mv.center_factor(R, "bf16", layout="tn")
    Lf, _, _, _ = mv.center_factor(R, "f32", layout="tn")
    Rt = float(np.percentile(mu.cpu().numpy(), 60))
    rsv = mv.RefinedSolver(Lb, Lf, mu, Rt, T, dtype="bf16", layout="tn", eps=1e-6)
    x, info = rsv.solve()
    assert info["converged"] == 1 and info["kkt"] <= 1e-6
    L64 = held(mv, Lf, None, n, "f32")
    ref = oracle_solution(L64, mu.cpu().numpy(), Rt)
    assert np.max(np.abs(x.cpu().numpy() - ref.x)) <= 1e-4


def test_tn_rejected_where_unsupported(mv):
    n, T = 64, 300
    R = gpu(panel(n, T, seed=3))
    Lt, _, mu, _ = mv.center_factor(R, "f32", layout="tn")
    p = mv.make_problem(Lt, mu, 0.0, T, layout="tn")
    assert mv.lib().mv_backward_workspace_size(mv.C.byref(p), None) == 0
    Lb, _, mub, _ = mv.center_factor(R, "bf16", layout="tn")
    pb = mv.make_problem(Lb, mub, 0.0, T, dtype="bf16", layout="tn")
    assert mv.lib().mv_frontier_workspace_size(mv.C.byref(pb), 4) == 0


@pytest.mark.parametrize("dt", ["f32", "fp8"])
@pytest.mark.parametrize("layout", ["nt", "tn"])
@pytest.mark.parametrize("shape", [(2000, 20000), (77, 300)])
def test_center_from_host_matches_device(mv, dt, layout, shape):
    """The chunked host-to-device pipeline gives the device call's bits (2000 x 20000: 3 chunks)."""
    n, T = shape
    R = torch.from_numpy(panel(n, T, seed=17)).pin_memory()
    L, rs, mu, tr = mv.center_factor(R.to(DEV), dt, layout=layout)
    Lh, rsh, muh, trh = mv.center_factor_host(R, dt, layout=layout, device=DEV)
    torch.cuda.synchronize()
    assert torch.equal(mu, muh)
    assert float(trh) == pytest.approx(float(tr), rel=1e-13)   # chunks slice the periods differently
    view = torch.uint8 if dt == "fp8" else L.dtype
    assert torch.equal(L.view(view), Lh.view(view))
    if dt == "fp8":
        assert torch.equal(rs, rsh)
