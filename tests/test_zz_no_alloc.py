"""mv_gradient_noalloc: the gradient for callers that may not allocate device
memory -- code that a host framework hands only input and output buffers
(the framework owns the device memory pool, as in plug-ins and user-defined
operators), or a latency-bound loop that cannot take the device-wide
synchronisation a cudaMalloc implies.

The entry point keeps its scratch in a fixed array inside the library, so
these checks call it through the C ABI twice in a row, with different inputs,
and compare each result element by element with the workspace-based
mv_gradient and with the FP64 oracle's gradient on the matrix the GPU holds,
at the tolerance the other gradient tests use (2e-5 relative to the largest
entry: FP32 accumulation over n or T terms).  Both storage layouts, the call
without z, the Python wrapper and the full 5440 x 48374 FP32 problem are
covered.  The file sorts last so that a run stopping at the first failure has
run everything else first; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import CFG_FULL, CFG_SMALL, factor_returns
from oracle.npga import gradient as oracle_gradient

pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module")
def mv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02917_gb300 import mv as m
    m.lib()
    return m


def _noalloc(mv, prob, y, T, with_z=True):
    n = y.numel()
    z = torch.full((T,), float("nan"), dtype=torch.float32, device=y.device) if with_z else None
    g = torch.full((n,), float("nan"), dtype=torch.float64, device=y.device)
    st = mv.lib().mv_gradient_noalloc(C.byref(prob), C.c_void_p(y.data_ptr()),
                                      C.c_void_p(z.data_ptr()) if with_z else None, C.c_void_p(g.data_ptr()),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == mv.MV_OK, mv.status_string(st)
    torch.cuda.synchronize()
    return z, g


def _dequant(L, rs, n, T, dt, layout):
    """The n x T matrix the GPU holds, in FP64."""
    A = L[:n, :T] if layout == "nt" else L[:T, :n].t()
    if dt == "f32":
        return A.double().cpu().numpy()
    if dt == "bf16":
        return A.float().double().cpu().numpy()
    q = A.cpu().view(torch.float8_e4m3fn).float().double().numpy()
    return q * rs.double().cpu().numpy()[:, None]


def _close(a, ref):
    a = np.asarray(a, dtype=np.float64)
    return np.max(np.abs(a - ref)) <= TOL * np.max(np.abs(ref))


CASES = [("f32", (333, 4999), "nt"), ("bf16", (200, 1000), "nt"), ("fp8", (2100, 9001), "nt"),
         ("f32", (200, 1000), "tn"), ("bf16", (1030, 4099), "tn")]


@pytest.mark.parametrize("dt,shape,layout", CASES)
def test_noalloc_gradient_matches_oracle_and_workspace_gradient_on_two_calls(mv, dt, shape, layout):
    n, T = shape
    R = factor_returns(CFG_SMALL.scaled(n, T, seed=5), np.float32)
    L, rs, mu, _ = mv.center_factor(torch.from_numpy(R).cuda(), dt, layout=layout)
    Lq = _dequant(L, rs, n, T, dt, layout)
    gamma = 3e-5
    prob = mv.make_problem(L, mu, 0.0, T, gamma, dt, rs, layout=layout)
    assert 0 < mv.lib().mv_gradient_noalloc_scratch_size(C.byref(prob)) <= mv.NOALLOC_SCRATCH_BYTES
    rng = np.random.default_rng(2)
    for call in range(2):                      # the second call must not see the first one's scratch
        y_h = rng.dirichlet(np.ones(n))
        y = torch.from_numpy(y_h).cuda()
        z_ref, g_ref = mv.gradient(L, y, T, gamma, dt, rs, layout=layout)
        z, g = _noalloc(mv, prob, y, T)
        z_o, g_o = Lq.T @ y_h, oracle_gradient(Lq, gamma, y_h)
        assert _close(z.double().cpu().numpy(), z_o) and _close(g.cpu().numpy(), g_o)
        assert _close(z.double().cpu().numpy(), z_ref.double().cpu().numpy())
        assert _close(g.cpu().numpy(), g_ref.cpu().numpy())
        # without z (d_z NULL) the same g
        _, g2 = _noalloc(mv, prob, y, T, with_z=False)
        assert np.array_equal(g2.cpu().numpy(), g.cpu().numpy())


def test_noalloc_python_wrapper(mv):
    n, T = 300, 2000
    R = factor_returns(CFG_SMALL.scaled(n, T, seed=6), np.float32)
    for layout in ("nt", "tn"):
        L, rs, mu, _ = mv.center_factor(torch.from_numpy(R).cuda(), "f32", layout=layout)
        y_h = np.random.default_rng(3).dirichlet(np.ones(n))
        y = torch.from_numpy(y_h).cuda()
        z, g = mv.gradient_noalloc(L, y, T, 1e-5, layout=layout)
        z_ref, g_ref = mv.gradient(L, y, T, 1e-5, layout=layout)
        assert _close(g.cpu().numpy(), g_ref.cpu().numpy()) and _close(z.double().cpu().numpy(),
                                                                       z_ref.double().cpu().numpy())
        _, g2 = mv.gradient_noalloc(L, y, T, 1e-5, layout=layout, with_z=False)
        assert np.array_equal(g2.cpu().numpy(), g.cpu().numpy())
        with pytest.raises(ValueError):
            mv.gradient_noalloc(L, y.float(), T, layout=layout)        # y must be FP64


@pytest.mark.slow
@pytest.mark.parametrize("layout", ["tn", "nt"])
def test_noalloc_full_size(mv, layout):
    """5440 x 48374 FP32 (1.05 GB): fits the fixed array; element-wise against the oracle."""
    n, T = CFG_FULL.n, CFG_FULL.T
    R = factor_returns(CFG_FULL, np.float32)
    L, _, mu, _ = mv.center_factor(torch.from_numpy(R).cuda(), "f32", layout=layout)
    del R
    prob = mv.make_problem(L, mu, 0.0, T, 0.0, "f32", None, layout=layout)
    need = mv.lib().mv_gradient_noalloc_scratch_size(C.byref(prob))
    assert 0 < need <= mv.NOALLOC_SCRATCH_BYTES
    Lq = _dequant(L, None, n, T, "f32", layout)
    rng = np.random.default_rng(9)
    for call in range(2):
        y_h = rng.dirichlet(np.ones(n))
        z, g = _noalloc(mv, prob, torch.from_numpy(y_h).cuda(), T)
        z_o = Lq.T @ y_h
        g_o = 2.0 * (Lq @ z_o)
        assert _close(z.double().cpu().numpy(), z_o) and _close(g.cpu().numpy(), g_o)


def test_noalloc_rejects_problems_beyond_its_scratch(mv):
    # Checked on the host before any launch, so fake aligned pointers suffice.
    p = mv.Problem()
    p.L, p.mu, p.n, p.T, p.ld, p.dtype = 4096, 4096, 32768, 1 << 20, 1 << 20, mv.MV_F32
    assert mv.lib().mv_gradient_noalloc_scratch_size(C.byref(p)) > mv.NOALLOC_SCRATCH_BYTES
    st = mv.lib().mv_gradient_noalloc(C.byref(p), C.c_void_p(4096), None, C.c_void_p(4096), None)
    assert st == mv.MV_ERR_UNSUPPORTED
    assert "bytes of scratch" in mv.lib().mv_last_error().decode()
