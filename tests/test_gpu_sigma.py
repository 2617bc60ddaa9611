"""GPU parity of the explicit-covariance path (Sec. 3 remark: NPGA with
grad f = 2 Sigma y + 2 gamma y).

* Formation: the GPU's Sigma against the FP64 product L_q L_q^T of the
  factor the GPU holds, entry by entry, within a bound derived from the
  arithmetic, in units of (|L_q| |L_q|^T)_ij and u = 2^-24: the tensor core
  accumulates at most 64 MMAs (1024 k-columns) into one FP32 partial, losing
  up to about an ulp of the partial per MMA (128 u); the nc partials
  (nc = ceil(T / 64) / 5 for FP32 L, ceil(T / 64) / 16 else) are added in FP32 with
  round-to-nearest (nc u); for FP32 L the BF16 hi/lo split drops terms below
  3 * 2^-18; for FP8 the row-scale product adds two roundings.  Sigma must
  be exactly symmetric.  Before partials were promoted to registers the
  FP32 diagonal at T = 48374 came out 4e-4 low: that bias is what the
  bound excludes.
* Product: Sigma y against the oracle's FP64 product with the downloaded
  Sigma (FP32 tile sums: 2e-5 of the largest entry), with NaN written into
  the padding columns past n, which must never be read.
* Solve: NPGA on the GPU's Sigma against oracle.npga_sigma on the same
  (downloaded) Sigma with the same step; x within 1e-4, objective within
  1e-5 relative, and the factor-form solve of the same problem lands on
  the same point.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import CFG_FULL, CFG_SMALL, factor_returns, power_start
from oracle.npga import initial_point, npga_sigma, objective_sigma, power_norm2_sigma, step_size

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
U = 2.0 ** -24


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


def held(L, rs, n, T, dt):
    """The n x T matrix the GPU holds (FP64)."""
    if dt == "f32":
        q = L[:, :T].double()
    elif dt == "bf16":
        q = L[:, :T].float().double()
    else:
        q = L[:, :T].cpu().view(torch.float8_e4m3fn).float().double()
    q = q.cpu().numpy()
    if dt == "fp8":
        q = q * rs.double().cpu().numpy()[:, None]
    return q


def form_rel(T, dt):
    # FP32: three products per k-step, chunks of 5 k-steps (60 MMAs); else chunks of 16 (64 MMAs)
    nc = -(-(-(-T // 64)) // (5 if dt == "f32" else 16))
    rel = (128 + nc + 16) * U
    if dt == "f32":
        rel += 3.0 * 2.0 ** -18
    if dt == "fp8":
        rel += 4.0 * U
    return rel


def form_bound(Lq, T, dt):
    A = np.abs(Lq)
    return form_rel(T, dt) * (A @ A.T) + 1e-30


@pytest.mark.parametrize("dt", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("shape", [(7, 50), (129, 1000), (300, 4099), (1030, 2011), (2100, 6007)])
def test_sigma_form_parity(mv, dt, shape):
    n, T = shape
    R = gpu(panel(n, T, seed=n + 1))
    L, rs, mu, tr = mv.center_factor(R, dt)
    S = mv.sigma_form(L, T, dt, rs)
    assert S.shape[0] == n and S.shape[1] % 4 == 0
    Sg = S[:, :n].double().cpu().numpy()
    assert np.array_equal(Sg, Sg.T)                          # exactly symmetric
    Lq = held(L, rs, n, T, dt)
    ref = Lq @ Lq.T
    err = np.abs(Sg - ref)
    assert np.all(err <= form_bound(Lq, T, dt))
    # trace of Sigma = ||L||_F^2 (the centering's FP64 trace is of the FP32 L)
    if dt == "f32":
        assert np.trace(Sg) == pytest.approx(float(tr), rel=1e-5)
    S2 = mv.sigma_form(L, T, dt, rs)
    assert torch.equal(S[:, :n], S2[:, :n])                  # deterministic


def test_sigma_form_rejects_bad_input(mv):
    R = gpu(panel(64, 300, seed=2))
    Lt, _, mu, _ = mv.center_factor(R, "f32", layout="tn")
    p = mv.make_problem(Lt, mu, 0.0, 300, layout="tn")
    assert mv.lib().mv_sigma_workspace_size(mv.C.byref(p)) == 0
    L, _, mu, _ = mv.center_factor(R, "f32")
    p = mv.make_problem(L, mu, 0.0, 300)
    S = torch.empty((64, 62), dtype=torch.float32, device=DEV)   # ldS < n
    st = mv.lib().mv_sigma_form(mv.C.byref(p), S.data_ptr(), 62, None, 0, None)
    assert st == mv.MV_ERR_INVALID_ARG


@pytest.mark.parametrize("n", [1, 2, 7, 128, 129, 300, 1031, 5440])
def test_sigma_product_parity(mv, n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n + 8))
    S64 = (A @ A.T) / (n + 8)
    ld = (n + 3) // 4 * 4 + 4
    S = torch.full((n, ld), float("nan"), dtype=torch.float32, device=DEV)   # NaN padding must not be read
    S[:, :n] = gpu(S64.astype(np.float32))
    Sq = S[:, :n].double().cpu().numpy()
    y = rng.dirichlet(np.ones(n)) if n > 1 else np.ones(1)
    gamma = 3e-3
    _, g = mv.gradient(S, gpu(y), 1, gamma, layout="sigma", with_z=False)
    g = g.cpu().numpy()
    ref = 2.0 * (Sq @ y) + 2.0 * gamma * y
    assert np.all(np.isfinite(g))
    assert np.max(np.abs(g - ref)) <= 2e-5 * np.max(np.abs(ref))
    _, g2 = mv.gradient(S, gpu(y), 1, gamma, layout="sigma", with_z=False)
    assert np.array_equal(g, g2.cpu().numpy())              # fixed-order reduction


@pytest.mark.parametrize("case", [(300, 2000, 0.0, "ge", 60), (1100, 4500, 2e-5, "eq", 40),
                                  (2100, 9001, 0.0, "ge", 70)])
def test_sigma_npga_parity(mv, case):
    n, T, gamma, mode, pct = case
    R = gpu(panel(n, T, seed=n + 5, base=CFG_FULL))
    L, _, mu, _ = mv.center_factor(R, "f32")
    S = mv.sigma_form(L, T, "f32")
    Sq = S[:, :n].double().cpu().numpy()
    mu_o = mu.cpu().numpy()
    Rt = float(np.percentile(mu_o, pct))
    r0 = power_start(n)
    x, info = mv.npga_solve(S, mu, Rt, T, gamma=gamma, mode=mode, eps=1e-6, power_start=gpu(r0),
                            layout="sigma")
    assert info["fused"] == 2
    assert info["converged"] == 1 and info["status"] == 0 and info["kkt"] <= 1e-6
    lam = power_norm2_sigma(Sq, r0, 50)
    assert info["lambda_hat"] == pytest.approx(lam, rel=1e-5)
    x = x.cpu().numpy()
    ref = npga_sigma(Sq, gamma, mu_o, Rt, initial_point(mu_o, Rt, mode), step_size(lam, gamma), eps=1e-11,
                     max_iter=200000, mode=mode)
    assert np.max(np.abs(x - ref.x)) <= 1e-4
    f = objective_sigma(Sq, gamma, x)
    assert (f - ref.f) / ref.f <= 1e-5
    assert info["objective"] == pytest.approx(f, rel=1e-5)
    # the factor form of the same problem reaches the same point
    xf, infof = mv.npga_solve(L, mu, Rt, T, gamma=gamma, mode=mode, eps=1e-6, power_start=gpu(r0))
    assert infof["converged"] == 1
    assert np.max(np.abs(xf.cpu().numpy() - x)) <= 2e-4


def test_sigma_full_size_sampled(mv):
    """5440 x 48374 FP32 (the full model): sampled rows of Sigma against FP64
    dot products of the held rows, exact symmetry, and one solve."""
    n, T = 5440, 48374
    R = gpu(panel(n, T, seed=1, base=CFG_FULL))
    L, _, mu, _ = mv.center_factor(R, "f32")
    del R
    S = mv.sigma_form(L, T, "f32")
    rows = np.array([0, 1, 127, 128, 2719, 4095, 5311, 5439])
    Lh = L[:, :T].cpu().numpy().astype(np.float64)    # the held FP32 values, FP64 products on the host
    Ah = np.abs(Lh)
    Sr = S[rows, :n].double().cpu().numpy()
    for k, i in enumerate(rows):
        ref = Lh @ Lh[i]
        scale = Ah @ Ah[i]
        assert np.all(np.abs(Sr[k] - ref) <= form_rel(T, "f32") * scale)
    assert torch.equal(S[:, :n], S[:, :n].t())
    Rt = float(np.percentile(mu.cpu().numpy(), 60))
    x, info = mv.npga_solve(S, mu, Rt, T, eps=1e-6, layout="sigma")
    assert info["converged"] == 1 and info["kkt"] <= 1e-6
    assert abs(x.sum().item() - 1.0) < 1e-9 and x.min().item() >= 0.0
