"""GPU parity of the uneven batch (mv_npga_solve_batch): independent problems
of different n and T, each from the small-config generator with its own
seed, solved together (grouped GEMV launches, one cluster per problem) and
compared one by one with the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import CFG_SMALL, factor_returns, power_start, uneven_problem_sizes
from oracle.center import center_factor
from oracle.npga import initial_point, kkt_residual, npga, objective, power_norm2, step_size

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02917_gb300 import mv as m
    m.lib()
    return m


def oracle_opt(L64, mu, Rt, gamma=0.0):
    lam = power_norm2(L64, power_start(L64.shape[0]), 300)
    return npga(L64, gamma, mu, Rt, initial_point(mu, Rt), step_size(lam, gamma), eps=1e-11, max_iter=200000)


def make(mv, models, dtype="f32", gammas=None):
    probs, host = [], []
    for j, m in enumerate(models):
        R = factor_returns(m, np.float32)
        L, rs, mu, _ = mv.center_factor(torch.from_numpy(R).cuda(), dtype)
        mu_o, L_o, _ = center_factor(R.astype(np.float64))
        Rt = float(np.percentile(mu_o, 55 + 5 * (j % 5)))
        g = 0.0 if gammas is None else gammas[j]
        probs.append({"L": L, "mu": mu, "R_target": Rt, "T": m.T, "row_scale": rs, "gamma": g})
        host.append((L_o, mu_o, Rt, g))
    return probs, host


def test_batch_uneven_parity(mv):
    shapes = [(150, 600), (900, 4000), (333, 1777), (512, 2048), (77, 3001), (640, 900)]
    models = [CFG_SMALL.scaled(n, T, seed=900 + j) for j, (n, T) in enumerate(shapes)]
    gammas = [0.0, 0.0, 2e-5, 0.0, 0.0, 1e-5]
    probs, host = make(mv, models, gammas=gammas)
    bs = mv.BatchSolver(probs, eps=1e-7)
    xs, infos = bs.solve()
    iters = set()
    for j, (x, info, (L_o, mu_o, Rt, g)) in enumerate(zip(xs, infos, host)):
        assert info["converged"] == 1, (j, info)
        x = x.cpu().numpy()
        ref = oracle_opt(L_o, mu_o, Rt, g)
        assert np.max(np.abs(x - ref.x)) <= 1e-4
        f = objective(L_o, g, x)
        assert (f - ref.f) / ref.f <= 1e-5
        assert info["objective"] == pytest.approx(f, rel=1e-5)
        assert kkt_residual(L_o, g, mu_o, Rt, x, info["alpha"]) <= 1.05e-7
        iters.add(info["iterations"])
    assert len(iters) > 1          # problems stop independently


def test_batch_matches_single_solves(mv):
    """Same iterates as one-at-a-time mv_npga_solve up to FP32 summation order
    (the batch splits the rows of L^T y differently)."""
    models = [CFG_SMALL.scaled(n, T, seed=950 + j) for j, (n, T) in enumerate([(200, 1000), (450, 2500)])]
    probs, host = make(mv, models)
    xs, infos = mv.BatchSolver(probs, eps=1e-6).solve()
    for q, x, info in zip(probs, xs, infos):
        xs1, i1 = mv.npga_solve(q["L"], q["mu"], q["R_target"], q["T"], eps=1e-6)
        assert abs(i1["iterations"] - info["iterations"]) <= 5
        assert torch.max(torch.abs(xs1 - x)).item() <= 1e-6


@pytest.mark.slow
def test_batch_uneven_config_sample(mv):
    """32 problems drawn from the 256-problem recipe (n ~ U[500,5000], T ~ U[2000,20000]); 3 checked."""
    models = uneven_problem_sizes()[:32]
    probs, host = make(mv, models)
    xs, infos = mv.BatchSolver(probs, eps=1e-6).solve()
    assert all(i["converged"] == 1 for i in infos)
    for j in (0, 7, 31):
        L_o, mu_o, Rt, g = host[j]
        x = xs[j].cpu().numpy()
        assert kkt_residual(L_o, g, mu_o, Rt, x, infos[j]["alpha"]) <= 1.05e-6
        assert x.min() >= 0 and abs(x.sum() - 1) < 1e-12 and mu_o @ x >= Rt - 1e-15


def test_batch_tiles_tuned_and_equivalent(mv):
    """The first solve of a batch shape tunes the grouped GEMV tiles; every
    candidate gives the same answer up to FP32 summation order."""
    models = [CFG_SMALL.scaled(n, T, seed=970 + j) for j, (n, T) in enumerate([(300, 2500), (700, 1200), (90, 4000)])]
    probs, host = make(mv, models)
    bs = mv.BatchSolver(probs, eps=1e-7)
    t_rows, n_bytes, tuned = bs.tiles()
    assert not tuned and (t_rows, n_bytes) == (512, 16384)
    xs, infos = bs.solve()
    t_rows, n_bytes, tuned = bs.tiles()
    assert tuned and t_rows in (256, 512, 1024) and n_bytes in (8192, 16384, 32768)
    xs = [x.clone() for x in xs]
    xs2, _ = bs.solve()                                  # cached choice, same bits
    assert all(torch.equal(a, b) for a, b in zip(xs, xs2))
    for x, info, (L_o, mu_o, Rt, g) in zip(xs, infos, host):
        assert info["converged"] == 1
        ref = oracle_opt(L_o, mu_o, Rt, g)
        assert np.max(np.abs(x.cpu().numpy() - ref.x)) <= 1e-4
