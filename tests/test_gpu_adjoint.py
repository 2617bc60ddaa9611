"""GPU adjoint of the unrolled NPGA solve (mv_npga_backward, FP32) against the
FP64 oracle adjoint on the same FP32 factor, step and start, and against
central finite differences of the oracle's FP64 forward (h = 1e-4 times the
RMS of each variable, 32 directions; directions whose +-h forwards change an
active set are kinks and are skipped).  The loss is the negative Sharpe-like
ratio of the returned portfolio on a held-out block of periods.

Tolerances.  d mu and d L are compared element by element, relative to the
largest entry of the oracle's gradient.  Every product of the GPU's forward
and reverse sweeps is one pass over L with FP32 terms and compensated
per-row sums, good to a few units of 2^-24 relative; the reverse recursion
applies projectors (the projection's Jacobian) and the contraction
I - 2 alpha L L^T to those errors, so they do not grow with K.  The dL
update of a segment is one tensor-core GEMM over three-piece BF16 splits:
its 6 x 2C piece products (768 k-columns, 48 MMA instructions) accumulate in
the FP32 tensor-memory accumulator, which drops up to an ulp of the running
sum per instruction, and the K / C segment results add into dL in FP32.
Measured: d mu 4e-8 and d L 1.2e-6 of the largest entry at K = 100, d L
1.7e-6 at K = 500; ADJ_TOL = 1e-5 (48 ulps of 2^-24 on each of the ten
segment sums, with room).  The directional derivative sums n T products of
d L with a random direction, whose cancellation magnifies the relative error
(up to 1.25e-5 measured); the finite-difference check, whose own truncation
error (h = 1e-4 of each variable's RMS: O(h^2) = 1e-8) and rounding error
(1e-16 / h of the loss) are far smaller, uses FD_TOL = 1e-4.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import CFG_SMALL, factor_returns
from oracle.center import center_factor
from oracle.npga import initial_point
from oracle import adjoint

pytestmark = pytest.mark.gpu

ADJ_TOL = 1e-5
FD_TOL = 1e-4


def max_rel(a, ref):
    """Largest element-wise error relative to the largest entry of ref."""
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


@pytest.fixture(scope="module")
def mv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02917_gb300 import mv as m
    m.lib()
    return m


def setup(mv, n, T, Ttest, seed, pct=60):
    R = factor_returns(CFG_SMALL.scaled(n, T + Ttest, seed=seed), np.float32)
    Rtr = np.ascontiguousarray(R[:, :T])
    L, _, mu, _ = mv.center_factor(torch.from_numpy(Rtr).cuda(), "f32")
    mu_o, _, _ = center_factor(Rtr.astype(np.float64))
    mu_t, L_t, _ = center_factor(R[:, T:].astype(np.float64))
    Rt = float(np.percentile(mu_o, pct))
    return L, mu, mu_o, mu_t, L_t, Rt


@pytest.mark.parametrize("K,C,mode", [(100, 20, "ge"), (100, 30, "ge"), (60, 25, "eq")])
def test_adjoint_parity_and_finite_differences(mv, K, C, mode):
    n, T, Ttest = 300, 1500, 400
    L, mu, mu_o, mu_t, L_t, Rt = setup(mv, n, T, Ttest, seed=81)
    x, info = mv.npga_solve(L, mu, Rt, T, mode=mode, eps=0.0, kkt_every=0, max_iter=K)
    alpha = info["alpha"]
    xK = x.cpu().numpy()
    L64 = L[:, :T].double().cpu().numpy()
    x0 = initial_point(mu_o, Rt, mode)
    xo, tape, betas = adjoint.unrolled_forward(L64, 0.0, mu_o, Rt, x0, alpha, K, mode, record=True)
    assert np.max(np.abs(xK - xo)) <= 1e-6                         # same forward
    gx = adjoint.sharpe_loss_grad(xo, mu_t, L_t)
    dmu, dL, binfo = mv.npga_backward(L, mu, Rt, T, torch.from_numpy(gx).cuda(), K, mode=mode,
                                      checkpoint_every=C)
    assert binfo["iterations"] == K and binfo["alpha"] == alpha
    mub_o, Lb_o = adjoint.backward(L64, 0.0, mu_o, alpha, tape, betas, gx)
    dmu = dmu.cpu().numpy()
    dL = dL[:, :T].double().cpu().numpy()
    e_mu, e_L = max_rel(dmu, mub_o), max_rel(dL, Lb_o)
    print(f"adjoint K={K} C={C} {mode}: d mu {e_mu:.2e}, d L {e_L:.2e} (element-wise, of max)")
    assert e_mu <= ADJ_TOL and e_L <= ADJ_TOL
    # central differences of the FP64 forward on random directions
    loss = lambda xx: adjoint.sharpe_loss(xx, mu_t, L_t)
    rng = np.random.default_rng(3)
    h = 1e-4
    rms_mu, rms_L = np.sqrt(np.mean(mu_o ** 2)), np.sqrt(np.mean(L64 ** 2))
    checked = 0
    worst = 0.0
    for _ in range(32):
        dm = rng.standard_normal(n)
        dm *= rms_mu / np.linalg.norm(dm)
        dD = rng.standard_normal(L64.shape)
        dD *= rms_L / np.linalg.norm(dD)
        _, tp, _ = adjoint.unrolled_forward(L64 + h * dD, 0.0, mu_o + h * dm, Rt, x0, alpha, K, mode, record=True)
        _, tm, _ = adjoint.unrolled_forward(L64 - h * dD, 0.0, mu_o - h * dm, Rt, x0, alpha, K, mode, record=True)
        kink = any(not np.array_equal(a["x1"] > 0, b["x1"] > 0) or not np.array_equal(a["x1"] > 0, c["x1"] > 0)
                   for a, b, c in zip(tape, tp, tm))
        if kink:
            continue
        fd = (loss(tp[-1]["x1"]) - loss(tm[-1]["x1"])) / (2 * h)
        an = dmu @ dm + np.sum(dL * dD)
        worst = max(worst, abs(an - fd) / abs(fd))
        assert an == pytest.approx(fd, rel=FD_TOL, abs=1e-10)
        checked += 1
    print(f"finite differences: {checked} directions, worst relative error {worst:.2e}")
    assert checked >= 16


def test_autograd_function_matches_backward(mv):
    n, T, Ttest, K = 200, 800, 300, 40
    L, mu, mu_o, mu_t, L_t, Rt = setup(mv, n, T, Ttest, seed=82)
    Lg = L.clone().requires_grad_(True)
    mug = mu.clone().requires_grad_(True)
    x = mv.NPGAFunction.apply(Lg, mug, Rt, T, K)
    mt = torch.from_numpy(mu_t).cuda()
    Lt = torch.from_numpy(L_t).cuda()
    loss = -(mt @ x) / torch.linalg.norm(Lt.T @ x)
    loss.backward()
    gx = adjoint.sharpe_loss_grad(x.detach().cpu().numpy(), mu_t, L_t)
    dmu, dL, _ = mv.npga_backward(L, mu, Rt, T, torch.from_numpy(gx).cuda(), K)
    assert torch.allclose(mug.grad, dmu, rtol=1e-6, atol=1e-12)
    assert torch.allclose(Lg.grad, dL, rtol=1e-5, atol=1e-9)


@pytest.mark.slow
def test_adjoint_full_config(mv):
    """2000 assets x 10000 periods (+2000 test), 500 iterations, checkpoints every 50."""
    n, T, Ttest, K = 2000, 10000, 2000, 500
    L, mu, mu_o, mu_t, L_t, Rt = setup(mv, n, T, Ttest, seed=0)
    x, info = mv.npga_solve(L, mu, Rt, T, eps=0.0, kkt_every=0, max_iter=K)
    alpha = info["alpha"]
    L64 = L[:, :T].double().cpu().numpy()
    x0 = initial_point(mu_o, Rt)
    xo, tape, betas = adjoint.unrolled_forward(L64, 0.0, mu_o, Rt, x0, alpha, K, record=True)
    assert np.max(np.abs(x.cpu().numpy() - xo)) <= 1e-5
    gx = adjoint.sharpe_loss_grad(xo, mu_t, L_t)
    dmu, dL, _ = mv.npga_backward(L, mu, Rt, T, torch.from_numpy(gx).cuda(), K, checkpoint_every=50)
    mub_o, Lb_o = adjoint.backward(L64, 0.0, mu_o, alpha, tape, betas, gx)
    dL = dL[:, :T].double().cpu().numpy()
    e_mu, e_L = max_rel(dmu.cpu().numpy(), mub_o), max_rel(dL, Lb_o)
    print(f"adjoint 2000x10000 K=500: d mu {e_mu:.2e}, d L {e_L:.2e} (element-wise, of max)")
    assert e_mu <= ADJ_TOL and e_L <= ADJ_TOL
