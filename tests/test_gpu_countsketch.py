"""GPU parity of the CountSketch map (Sec. 2.3, construction (2)).

tilde L = L Phi with Phi(t, h(t)) = s_t.  The GPU sums each bucket's
periods in ascending order in FP32; against the oracle's FP64 product on
the factor the GPU holds the error of entry (i, j) is at most
(k_j + 2) u sum_{t in bucket j} |L_it| (k_j periods in the bucket,
u = 2^-24; FP8 adds the row-scale multiplication).  Both layouts, all three
storage types, ragged shapes, empty buckets (m > T), the full 5440 x 48374
workload on sampled rows, and the STR truncation fed by this sketch.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import CFG_FULL, CFG_SMALL, countsketch_hash, factor_returns
from oracle import strmodel

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


def held_nt(L, rs, n, T, dt, layout):
    """The n x T matrix the GPU holds (FP64), from either layout."""
    M = L[:, :T] if layout == "nt" else L[:T, :n]
    if dt == "fp8":
        q = M.cpu().view(torch.float8_e4m3fn).float().double().numpy()
    else:
        q = M.float().double().cpu().numpy()
    if layout == "tn":
        q = q.T
    if dt == "fp8":
        q = q * rs.double().cpu().numpy()[:, None]
    return q


def bound(Lq, h, m):
    A = np.abs(Lq) @ strmodel.countsketch_matrix(h, np.ones_like(h), m)     # sum of |terms| per bucket
    k = np.bincount(h, minlength=m).astype(np.float64)
    return (k[None, :] + 2.0) * U * A + 1e-30


@pytest.mark.parametrize("layout", ["tn", "nt"])
@pytest.mark.parametrize("dt", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("shape", [(7, 50, 13), (300, 4099, 512), (1030, 2011, 8192), (2100, 6007, 1000)])
def test_countsketch_parity(mv, layout, dt, shape):
    n, T, m = shape
    R = gpu(factor_returns(CFG_SMALL.scaled(n, T, seed=n + 7), np.float32))
    L, rs, _, _ = mv.center_factor(R, dt, layout=layout)
    h, sg = countsketch_hash(T, m, seed=T)
    out = mv.countsketch(L, n, T, gpu(h), gpu(sg), m, dt, rs, layout)
    Lq = held_nt(L, rs, n, T, dt, layout)
    ref = strmodel.countsketch(Lq, h, sg, m)
    got = out[:, :m].double().cpu().numpy()
    assert np.all(np.abs(got - ref) <= bound(Lq, h, m) * (2.0 if dt == "fp8" else 1.0))
    empty = np.bincount(h, minlength=m) == 0
    assert np.all(got[:, empty] == 0.0)
    out2 = mv.countsketch(L, n, T, gpu(h), gpu(sg), m, dt, rs, layout)
    assert torch.equal(out, out2)                            # deterministic


def test_countsketch_layouts_agree_bitwise(mv):
    """Both layouts sum each bucket in ascending period order: identical bits."""
    n, T, m = 777, 5003, 640
    R = gpu(factor_returns(CFG_SMALL.scaled(n, T, seed=3), np.float32))
    h, sg = countsketch_hash(T, m, seed=9)
    Ln, _, _, _ = mv.center_factor(R, "f32", layout="nt")
    Lt, _, _, _ = mv.center_factor(R, "f32", layout="tn")
    a = mv.countsketch(Ln, n, T, gpu(h), gpu(sg), m, "f32", None, "nt")
    b = mv.countsketch(Lt, n, T, gpu(h), gpu(sg), m, "f32", None, "tn")
    assert torch.equal(a, b)


def test_countsketch_rejects_bad_bucket(mv):
    n, T, m = 64, 300, 32
    R = gpu(factor_returns(CFG_SMALL.scaled(n, T, seed=3), np.float32))
    L, _, _, _ = mv.center_factor(R, "f32", layout="tn")
    h, sg = countsketch_hash(T, m, seed=1)
    h[17] = m                                                # out of range: the kernels skip it and report
    with pytest.raises(mv.MvError) as e:
        mv.countsketch(L, n, T, gpu(h), gpu(sg), m, "f32", None, "tn")
    assert e.value.status == mv.MV_ERR_INVALID_ARG


def test_countsketch_full_size_and_str(mv):
    """5440 x 48374 FP32 L^T, m = 8192: sampled rows against the oracle, then
    the truncation of this sketch: sigma^2 are the top eigenvalues of
    tilde L tilde L^T within 1e-5 sigma_1^2, the STR tests' tolerance (the
    truncation forms the Gram matrix from three-piece BF16 products to FP32
    accuracy, about 1e-6 sigma_1^2 on the eigenvalues, and solves its small
    Rayleigh--Ritz problem in FP64)."""
    n, T, m = 5440, 48374, 8192
    R = gpu(factor_returns(CFG_FULL, np.float32))
    Lt, _, _, _ = mv.center_factor(R, "f32", layout="tn")
    del R
    h, sg = countsketch_hash(T, m, seed=2)
    out = mv.countsketch(Lt, n, T, gpu(h), gpu(sg), m, "f32", None, "tn")
    rows = [0, 1, 2047, 2048, 4095, 5439]
    Lr = Lt[:T, rows].double().cpu().numpy().T                # held rows of L, FP64
    ref = strmodel.countsketch(Lr, h, sg, m)
    got = out[rows, :m].double().cpu().numpy()
    assert np.all(np.abs(got - ref) <= bound(Lr, h, m))
    Leff, sigma, gamma = mv.str_truncate(out[:, :m].contiguous(), 64)
    K = out[:, :m].double().cpu().numpy()
    lam = np.sort(np.linalg.eigvalsh(K @ K.T))[::-1][:64]
    s = sigma.cpu().numpy()
    assert np.max(np.abs(s ** 2 - lam)) <= 1e-5 * lam[0]


@pytest.mark.parametrize("layout", ["tn", "nt"])
def test_countsketch_many_buckets(mv, layout):
    """20000 buckets for 30011 periods (about 1.5 per bucket, many empty):
    the sums match the oracle and every empty bucket's column is zero."""
    n, T, m = 150, 30011, 20000
    R = gpu(factor_returns(CFG_SMALL.scaled(n, T, seed=41), np.float32))
    L, rs, _, _ = mv.center_factor(R, "f32", layout=layout)
    h, sg = countsketch_hash(T, m, seed=5)
    out = mv.countsketch(L, n, T, gpu(h), gpu(sg), m, "f32", rs, layout)
    Lq = held_nt(L, rs, n, T, "f32", layout)
    ref = strmodel.countsketch(Lq, h, sg, m)
    got = out[:, :m].double().cpu().numpy()
    assert np.all(np.abs(got - ref) <= bound(Lq, h, m))
    empty = np.bincount(h, minlength=m) == 0
    assert empty.any() and np.all(got[:, empty] == 0.0)


@pytest.mark.parametrize("m", [100, 20000])
def test_countsketch_crowded_bucket(mv, m):
    """One bucket of 3000 periods, sorted in place rather than by the
    16-input register network, beside short buckets (m = 20000) or beside
    buckets of about 240 periods (m = 100); both layouts give identical bits."""
    n, T = 96, 24007
    R = gpu(factor_returns(CFG_SMALL.scaled(n, T, seed=43), np.float32))
    h, sg = countsketch_hash(T, m, seed=8)
    h[5000:8000] = 7
    outs = []
    for layout in ("tn", "nt"):
        L, _, _, _ = mv.center_factor(R, "f32", layout=layout)
        out = mv.countsketch(L, n, T, gpu(h), gpu(sg), m, "f32", None, layout)
        Lq = held_nt(L, None, n, T, "f32", layout)
        ref = strmodel.countsketch(Lq, h, sg, m)
        got = out[:, :m].double().cpu().numpy()
        assert np.all(np.abs(got - ref) <= bound(Lq, h, m))
        outs.append(out)
    assert torch.equal(outs[0], outs[1])
