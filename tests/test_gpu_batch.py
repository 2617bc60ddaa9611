"""GPU parity of the uneven batch (mv_npga_solve_batch): independent problems
of different n and T, each from the small-config generator with its own
seed, solved together (grouped GEMV launches, one cluster per problem) and
compared one by one with the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import CFG_SMALL, factor_returns, power_start, uneven_problem_sizes
from oracle.center import center_factor
from oracle.npga import (fw_gap, initial_point, kkt_residual, npga, npga_sigma, objective, objective_sigma,
                         power_norm2, power_norm2_sigma, sigma_from_factor, step_size)

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


def make(mv, models, dtype="f32", gammas=None, layouts=None):
    probs, host = [], []
    for j, m in enumerate(models):
        R = factor_returns(m, np.float32)
        lay = "nt" if layouts is None else layouts[j]
        L, rs, mu, _ = mv.center_factor(torch.from_numpy(R).cuda(), dtype, layout=lay)
        mu_o, L_o, _ = center_factor(R.astype(np.float64))
        Rt = float(np.percentile(mu_o, 55 + 5 * (j % 5)))
        g = 0.0 if gammas is None else gammas[j]
        probs.append({"L": L, "mu": mu, "R_target": Rt, "T": m.T, "row_scale": rs, "gamma": g, "layout": lay})
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


@pytest.mark.parametrize("layouts", ["tn", "mixed"])
def test_batch_transposed_parity(mv, layouts):
    """Problems stored L^T (T x n) take the grouped single pass: one launch
    per cluster size over (problem, cluster) pairs.  Sizes span one CTA per
    cluster (n <= 2816 FP32) and pairs (n = 3001), ragged n and T, tiny and
    large problems side by side; "mixed" puts n x T problems (grouped GEMVs)
    in the same batch.  Each against the FP64 oracle optimum."""
    shapes = [(150, 600), (3001, 4099), (333, 1777), (1024, 8192), (77, 3001), (2900, 900), (640, 20011)]
    models = [CFG_SMALL.scaled(n, T, seed=880 + j) for j, (n, T) in enumerate(shapes)]
    gammas = [0.0, 0.0, 2e-5, 0.0, 0.0, 1e-5, 0.0]
    lay = ["tn"] * len(shapes) if layouts == "tn" else ["tn", "nt"] * 3 + ["tn"]
    probs, host = make(mv, models, gammas=gammas, layouts=lay)
    bs = mv.BatchSolver(probs, eps=1e-7)
    xs, infos = bs.solve()
    for j, (x, info, (L_o, mu_o, Rt, g)) in enumerate(zip(xs, infos, host)):
        assert info["converged"] == 1, (j, info)
        x = x.cpu().numpy()
        ref = oracle_opt(L_o, mu_o, Rt, g)
        assert np.max(np.abs(x - ref.x)) <= 1e-4, j
        f = objective(L_o, g, x)
        assert (f - ref.f) / ref.f <= 1e-5, j
        assert info["objective"] == pytest.approx(f, rel=1e-5)
        assert kkt_residual(L_o, g, mu_o, Rt, x, info["alpha"]) <= 1.05e-7, j


@pytest.mark.parametrize("dt", ["bf16", "fp8"])
def test_batch_transposed_low_precision(mv, dt):
    """BF16 / FP8 factors stored transposed: the grouped pass against the
    single-problem solve on the same stored matrix (same kernels per
    problem, so the iterates agree to FP32 summation order)."""
    shapes = [(700, 5003), (2000, 4096), (300, 1000)]
    models = [CFG_SMALL.scaled(n, T, seed=860 + j) for j, (n, T) in enumerate(shapes)]
    probs, host = make(mv, models, dtype=dt, layouts=["tn"] * 3)
    xs, infos = mv.BatchSolver(probs, dtype=dt, eps=1e-6).solve()
    for q, x, info in zip(probs, xs, infos):
        assert info["converged"] == 1
        x1, i1 = mv.npga_solve(q["L"], q["mu"], q["R_target"], q["T"], dtype=dt, row_scale=q["row_scale"],
                               eps=1e-6, layout="tn")
        assert abs(i1["iterations"] - info["iterations"]) <= 5
        assert torch.max(torch.abs(x1 - x)).item() <= 1e-5


def test_batch_transposed_matches_nt(mv):
    """The same problems stored both ways give the same solutions."""
    models = [CFG_SMALL.scaled(n, T, seed=840 + j) for j, (n, T) in enumerate([(1200, 6000), (450, 2500)])]
    pn, _ = make(mv, models, layouts=["nt", "nt"])
    pt, _ = make(mv, models, layouts=["tn", "tn"])
    xn, inn = mv.BatchSolver(pn, eps=1e-7).solve()
    xn = [x.clone() for x in xn]
    xt, itn = mv.BatchSolver(pt, eps=1e-7).solve()
    for a, b, i, j in zip(xn, xt, inn, itn):
        assert i["converged"] == 1 and j["converged"] == 1
        assert torch.max(torch.abs(a - b)).item() <= 1e-6
        assert j["objective"] == pytest.approx(i["objective"], rel=1e-6)


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
@pytest.mark.parametrize("layout", ["tn", "nt"])
def test_batch_uneven_config_sample(mv, layout):
    """32 problems drawn from the 256-problem recipe (n ~ U[500,5000],
    T ~ U[2000,20000]) solved together to KKT 1e-6; four of them (the first,
    the last, one in between and the largest n) against the FP64 optimum:
    the oracle rounds its centred L to FP32 (the GPU's L, bit for bit), forms
    Sigma = L L^T and runs Algorithm 1 on it to KKT 1e-10.  x within 1e-4 of
    x* in the infinity norm, the objective within 1e-5 relative, and
    f(x) - f* bounded by the Frank--Wolfe gap at x (Sec. 5.2's gap metric)."""
    models = uneven_problem_sizes()[:32]
    probs, host = make(mv, models, layouts=[layout] * 32)
    xs, infos = mv.BatchSolver(probs, eps=1e-6).solve()
    assert all(i["converged"] == 1 for i in infos)
    big = int(np.argmax([m.n for m in models]))
    for j in sorted({0, 7, 31, big}):
        L_o, mu_o, Rt, g = host[j]
        L_o = L_o.astype(np.float32).astype(np.float64)
        x = xs[j].cpu().numpy()
        assert kkt_residual(L_o, g, mu_o, Rt, x, infos[j]["alpha"]) <= 1.05e-6
        assert x.min() >= 0 and abs(x.sum() - 1) < 1e-12 and mu_o @ x >= Rt - 1e-15
        Sig = sigma_from_factor(L_o)
        r0 = power_start(L_o.shape[0])
        ref = npga_sigma(Sig, g, mu_o, Rt, initial_point(mu_o, Rt),
                         step_size(power_norm2_sigma(Sig, r0, 100), g), eps=1e-10, max_iter=50000)
        assert ref.converged, j
        f = objective_sigma(Sig, g, x)
        assert np.max(np.abs(x - ref.x)) <= 1e-4, j
        assert (f - ref.f) / ref.f <= 1e-5, j
        assert infos[j]["objective"] == pytest.approx(f, rel=1e-5)
        assert -1e-14 * ref.f <= f - ref.f <= fw_gap(L_o, g, mu_o, Rt, x) + 1e-12 * ref.f, j


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
