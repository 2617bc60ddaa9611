"""mv_gradient_noalloc: the gradient for callers that may not allocate device
memory (for instance code that a host framework hands only input and output
buffers, because the framework owns the device memory pool).

The entry point keeps its scratch in a fixed array inside the library, so
these checks call it through the C ABI twice in a row, with different inputs,
and compare each result with the workspace-based mv_gradient at the tolerance
the other gradient tests use (2e-5 relative, FP32 accumulation).  The file
sorts last so that a run stopping at the first failure has run everything
else first; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import CFG_SMALL, factor_returns

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02917_gb300 import mv as m
    m.lib()
    return m


def _noalloc(mv, prob, y, T):
    n = y.numel()
    z = torch.full((T,), float("nan"), dtype=torch.float32, device=y.device)
    g = torch.full((n,), float("nan"), dtype=torch.float64, device=y.device)
    st = mv.lib().mv_gradient_noalloc(C.byref(prob), C.c_void_p(y.data_ptr()), C.c_void_p(z.data_ptr()),
                                      C.c_void_p(g.data_ptr()),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == mv.MV_OK, mv.status_string(st)
    torch.cuda.synchronize()
    return z, g


@pytest.mark.parametrize("dt,shape", [("f32", (333, 4999)), ("bf16", (200, 1000)), ("fp8", (2100, 9001))])
def test_noalloc_gradient_matches_workspace_gradient_on_two_calls(mv, dt, shape):
    n, T = shape
    R = factor_returns(CFG_SMALL.scaled(n, T, seed=5), np.float32)
    L, rs, mu, _ = mv.center_factor(torch.from_numpy(R).cuda(), dt)
    gamma = 3e-5
    prob = mv.make_problem(L, mu, 0.0, T, gamma, dt, rs)
    rng = np.random.default_rng(2)
    for call in range(2):                      # the second call must not see the first one's scratch
        y = torch.from_numpy(rng.dirichlet(np.ones(n))).cuda()
        z_ref, g_ref = mv.gradient(L, y, T, gamma, dt, rs)
        z, g = _noalloc(mv, prob, y, T)
        zr, gr = z_ref.double().cpu().numpy(), g_ref.cpu().numpy()
        assert np.max(np.abs(z.double().cpu().numpy() - zr)) <= 2e-5 * np.max(np.abs(zr))
        assert np.max(np.abs(g.cpu().numpy() - gr)) <= 2e-5 * np.max(np.abs(gr))


def test_noalloc_rejects_problems_beyond_its_scratch(mv):
    # Checked on the host before any launch, so fake aligned pointers suffice.
    p = mv.Problem()
    p.L, p.mu, p.n, p.T, p.ld, p.dtype = 4096, 4096, 32768, 1 << 20, 1 << 20, mv.MV_F32
    st = mv.lib().mv_gradient_noalloc(C.byref(p), C.c_void_p(4096), None, C.c_void_p(4096), None)
    assert st == mv.MV_ERR_UNSUPPORTED
    assert "bytes of scratch" in mv.lib().mv_last_error().decode()
