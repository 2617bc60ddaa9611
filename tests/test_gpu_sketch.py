"""GPU parity of the tcgen05 sketch GEMM (tilde L = L Phi, Sec. 2.3) against
the FP64 oracle on the same BF16 inputs.

FP32 accumulation over K terms: the error of entry (i, j) is bounded by a
small multiple of sqrt(K) 2^-24 sum_k |L_ik Phi_kj|; the tests use 1e-5 of
that magnitude sum (K <= 48374)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import CFG_FULL, CFG_SMALL, factor_returns, gaussian_sketch
from oracle import strmodel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02917_gb300 import mv as m
    m.lib()
    return m


def _case(mv, n, T, m, seed):
    R = factor_returns(CFG_SMALL.scaled(n, T, seed=seed), np.float32)
    L, _, _, _ = mv.center_factor(torch.from_numpy(R).cuda(), "bf16")
    Phi_t = mv.bf16_rows(gaussian_sketch(T, m, seed=seed + 1))
    Ls = mv.sketch(L, T, Phi_t)
    torch.cuda.synchronize()
    A = L[:, :T].float().double().cpu().numpy()
    B = Phi_t[:, :T].float().double().cpu().numpy()
    return Ls.double().cpu().numpy(), A, B


@pytest.mark.parametrize("shape", [(128, 64, 256), (300, 2000, 512), (77, 1000, 300), (1, 130, 8)])
def test_sketch_gemm_parity_small(mv, shape):
    n, T, m = shape
    Ls, A, B = _case(mv, n, T, m, seed=40 + n)
    ref = strmodel.sketch(A, B)
    mag = np.abs(A) @ np.abs(B).T
    assert Ls.shape == ref.shape
    assert np.all(np.abs(Ls - ref) <= 1e-5 * mag + 1e-30)


@pytest.mark.slow
def test_sketch_gemm_full_size_sampled(mv):
    """5440 x 48374 times 48374 x 8192 (4.31 TFLOP): sampled entries vs FP64 dot products."""
    m_ = CFG_FULL
    R = factor_returns(m_, np.float32)
    L, _, _, _ = mv.center_factor(torch.from_numpy(R).cuda(), "bf16")
    del R
    Phi_t = mv.bf16_rows(gaussian_sketch(m_.T, 8192, seed=2, dtype=np.float32))
    Ls = mv.sketch(L, m_.T, Phi_t)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    rows = rng.integers(0, m_.n, 64)
    cols = rng.integers(0, 8192, 64)
    rows[:4] = [0, m_.n - 1, 5376, 5439]      # first, last and last-tile rows
    cols[:4] = [0, 8191, 255, 256]
    A = L[torch.from_numpy(rows).cuda(), :m_.T].float().double().cpu().numpy()
    B = Phi_t[torch.from_numpy(cols).cuda(), :m_.T].float().double().cpu().numpy()
    got = Ls[torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()].double().cpu().numpy()
    ref = np.einsum("ij,ij->i", A, B)
    mag = np.einsum("ij,ij->i", np.abs(A), np.abs(B))
    assert np.all(np.abs(got - ref) <= 1e-5 * mag)
    # no systematic shrink: a one-sided accumulator rounding over the 3024 MMAs of
    # one output would scale every entry by about 1 - 5e-5 (the chunked accumulation
    # leaves one chunk's worth, about 5e-7)
    slope = float(got @ ref / (ref @ ref))
    assert abs(slope - 1.0) <= 5e-6, slope


# ------------------------------------------------------------------ seeded draws (rng.cuh vs oracle/rng.py)
@pytest.mark.parametrize("m,T,seed", [(64, 1001, 5), (300, 4096, 2 ** 40 + 7), (8192, 48374, 2)])
def test_gaussian_sketch_draw_matches_oracle(mv, m, T, seed):
    """mv_gaussian_sketch against the oracle's Philox4x32-10 + Box--Muller in
    FP64, rounded to BF16: bit-identical (the device evaluates the transform
    in FP32 and again in FP64 wherever the FP32 value lies near a BF16
    rounding midpoint, so it stores the correctly rounded value).  Padding
    columns are zero.  At the full 8192 x 48374 size, 64 rows are compared."""
    from oracle.rng import gaussian_sketch_bf16
    P = mv.gaussian_sketch(seed, m, T)
    torch.cuda.synchronize()
    rows = np.arange(m) if m <= 512 else np.r_[0, 1, m - 1, np.random.default_rng(1).integers(0, m, 61)]
    ref = gaussian_sketch_bf16(seed, m, T, rows=rows)
    got = P[torch.from_numpy(rows).cuda(), :T].double().cpu().numpy()
    assert np.array_equal(got, ref), f"{int(np.sum(got != ref))} of {got.size} entries differ"
    assert int(torch.count_nonzero(P[:, T:])) == 0


def test_countsketch_draw_matches_oracle(mv):
    """The hash and signs are integer functions of the Philox words: bit-exact."""
    from oracle.rng import countsketch_draw
    for T, m, seed in ((10007, 8192, 3), (48374, 1000, 2 ** 33 + 1)):
        h, sg = mv.countsketch_draw(seed, T, m)
        ho, so = countsketch_draw(seed, T, m)
        assert np.array_equal(h.cpu().numpy(), ho.astype(np.int32))
        assert np.array_equal(sg.cpu().numpy(), so)


# ------------------------------------------------------------------ FP32 and FP8 factors
@pytest.mark.parametrize("dt", ["f32", "fp8", "bf16"])
@pytest.mark.parametrize("shape", [(300, 2000, 512), (77, 1001, 300)])
def test_sketch_dtype_parity(mv, dt, shape):
    """tilde L = L Phi for a factor stored in FP32 (BF16 hi + lo split), FP8
    (exact BF16 expansion, row scales in the epilogue) or BF16, against the
    FP64 oracle on the matrix the GPU holds and the oracle's own draw of Phi
    (rounded to BF16, so exact in the BF16 upload).  FP32 adds the split's rounding, below 2^-18 |L_it|
    per term, to the FP32 accumulation bound of the BF16 test."""
    from oracle.rng import gaussian_sketch_bf16
    n, T, m = shape
    R = factor_returns(CFG_SMALL.scaled(n, T, seed=70 + n), np.float32)
    L, rs, _, _ = mv.center_factor(torch.from_numpy(R).cuda(), dt)
    B = gaussian_sketch_bf16(9, m, T)
    Phi_t = mv.bf16_rows(B)
    Ls = mv.sketch_dtype(L, T, Phi_t, dt, rs).double().cpu().numpy()
    if dt == "f32":
        A = L[:, :T].double().cpu().numpy()
    elif dt == "bf16":
        A = L[:, :T].float().double().cpu().numpy()
    else:
        A = L[:, :T].cpu().view(torch.float8_e4m3fn).float().double().numpy() * rs.double().cpu().numpy()[:, None]
    ref = strmodel.sketch(A, B)
    mag = np.abs(A) @ np.abs(B).T
    assert np.all(np.abs(Ls - ref) <= 1e-5 * mag + 1e-30)


@pytest.mark.parametrize("dt", ["bf16", "f32", "fp8"])
def test_sketch_str_from_seed(mv, dt):
    """mv_sketch_str draws Phi from its seed, sketches the factor of any type
    and truncates: the oracle draws the same Phi (oracle/rng.py, rounded to
    BF16), sketches the same matrix in FP64 and truncates by eigh.  Eigenvalues
    within 1e-5 sigma_1^2, L_eff^T L_eff = diag(sigma^2), eigen-residuals on
    the GPU's tilde L, and the ridge 1e-4 tr(Sigma) / n."""
    from oracle.rng import gaussian_sketch_bf16
    from oracle.center import center_factor
    n, T, m, k, seed = 300, 2000, 512, 64, 77
    R = factor_returns(CFG_SMALL.scaled(n, T, seed=71), np.float32)
    L, rs, _, tr = mv.center_factor(torch.from_numpy(R).cuda(), dt)
    L_eff, sigma, gamma, Ls = mv.sketch_str(L, T, m, seed, k, dt, rs, -1.0, float(tr.cpu()))
    torch.cuda.synchronize()
    if dt == "f32":
        A = L[:, :T].double().cpu().numpy()
    elif dt == "bf16":
        A = L[:, :T].float().double().cpu().numpy()
    else:
        A = L[:, :T].cpu().view(torch.float8_e4m3fn).float().double().numpy() * rs.double().cpu().numpy()[:, None]
    B = gaussian_sketch_bf16(seed, m, T)
    _, sig_o, _ = strmodel.truncate(strmodel.sketch(A, B), k)
    sig = sigma.cpu().numpy()
    s1 = sig_o[0] ** 2
    assert np.max(np.abs(sig ** 2 - sig_o ** 2)) <= 1e-5 * s1
    E = L_eff.double().cpu().numpy()
    assert np.max(np.abs(E.T @ E - np.diag(sig ** 2))) <= 1e-5 * s1
    Lt = Ls.double().cpu().numpy()
    for c in range(k):
        u = E[:, c] / sig[c]
        assert np.linalg.norm(Lt @ (Lt.T @ u) - sig[c] ** 2 * u) <= 1e-5 * s1
    tr_o = center_factor(R.astype(np.float64))[2]
    assert gamma == pytest.approx(1e-4 * tr_o / n, rel=1e-12)
