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
