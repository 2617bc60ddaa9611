"""Benchmark: NPGA time to a 1e-6 KKT residual at the paper's full shape.

Workload: n = 5440 assets x T = 48374 periods (the paper's real-data shape,
Sec. 5.2), synthetic 20-factor returns from ``synth.CFG_FULL`` (the paper's
panel is proprietary), centered on the GPU, L stored as FP32 (1.05 GB, far
larger than L2, so no flush is needed between steps).  One step = one full
solve through the C ABI: 50 power iterations for the step size, NPGA with a
KKT check every 5 iterations until the residual is <= 1e-6, and the final
objective.  Inputs are resident in HBM when the timed region starts.  L is
stored transposed (T x n) by default, where the fused single-pass product
L L^T y streams at copy speed; ``--layout nt`` keeps it n x T.

Printed JSON (one line, rank 0): value = seconds per solve (lower is
better), e2e = the same through host buffers (upload R, center, solve,
download x), roofline = the dominant gemv kernel's HBM throughput measured
with CUDA events around every launch of the loop, cpu_baseline = one complete
solve of the same workload by the FP64 oracle on this host's cores.

``--impl reference`` times the FP64 oracle (the CPU restatement of the
method) instead, as the reference arm.  Multi-GPU (torchrun): every rank
solves its own problem (replicas, no collective in the path); the time is
the max over ranks.
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-6 KKT, NPGA full model n=5440 T=48374"
FALLBACK_HBM = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mv", choices=["mv", "reference"])
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "fp8"])
    ap.add_argument("--layout", default="tn", choices=["tn", "nt"],
                    help="storage of L: tn = L^T (T x n, the fast layout), nt = n x T")
    ap.add_argument("--two-pass", action="store_true",
                    help="stream L twice per product (z = L^T y, then L z) instead of the fused single pass")
    ap.add_argument("--config", default="full", choices=["full", "small"])
    ap.add_argument("--eps", type=float, default=1e-6)
    ap.add_argument("--step-estimate", default="lanczos", choices=["lanczos", "power"],
                    help="lambda_hat for the fixed step (Sec. 3.1): Lanczos steps or power iterations on L L^T")
    ap.add_argument("--step-iters", type=int, default=None,
                    help="products spent on lambda_hat (default: 25 Lanczos steps, or 50 power iterations)")
    ap.add_argument("--shape", default=None, help="n,T override (profiling runs on a smaller case)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the BF16/FP8 + FP32-refinement lines")
    ap.add_argument("--no-str", action="store_true", help="skip the sketch / STR measurement")
    ap.add_argument("--sketch-m", type=int, default=8192)
    ap.add_argument("--no-frontier", action="store_true", help="skip the 64-target frontier measurement")
    ap.add_argument("--no-small", action="store_true", help="skip the 200 x 1000, 2000-iteration solve")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the 256-problem uneven batch")
    ap.add_argument("--no-sigma", action="store_true", help="skip the explicit-covariance measurement")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--str-k", type=int, default=512)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-row-oracles", action="store_true", help="skip the oracle timings of the further rows")
    ap.add_argument("--profile", default=None, choices=["sketch", "frontier", "batch", "str", "adjoint"],
                    help="run one instance of that workload at --shape (for ncu) and exit, printing its time")
    return ap.parse_args()


def step_opts(args):
    """Solver options of the step estimate, and its label."""
    if args.step_estimate == "lanczos":
        k = args.step_iters or 25
        return {"lanczos": 1, "power_iters": k}, f"{k} Lanczos steps"
    k = args.step_iters or 50
    return {"power_iters": k}, f"{k} power iterations"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value, world, device):
    """The largest of every rank's value (the whole job waits for its slowest rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(args, rank):
    from synth import CFG_FULL, CFG_SMALL
    base = CFG_FULL if args.config == "full" else CFG_SMALL
    n, T = base.n, base.T
    if args.shape:
        n, T = (int(v) for v in args.shape.split(","))
    # each rank solves its own independent problem (weak scaling)
    return base.scaled(n, T, seed=base.seed + rank)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


def jsonable(o, path="line"):
    """Plain JSON values; a stray 0-d tensor or NumPy scalar is converted (and reported)."""
    if isinstance(o, dict):
        return {k: jsonable(v, f"{path}.{k}") for k, v in o.items()}
    if isinstance(o, (list, tuple)):
        return [jsonable(v, f"{path}[{i}]") for i, v in enumerate(o)]
    if o is None or isinstance(o, (bool, int, float, str)):
        return o
    if hasattr(o, "item"):
        sys.stderr.write(f"bench: {path} was a {type(o).__name__}; converted\n")
        return o.item()
    return o


def peaks_tensor():
    """(dense BF16 tensor peak in TFLOP/s, "measured" | "fallback"): the burst
    figure (the GEMMs are timed alone), else the 1.9 PFLOP/s fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


# kernel -> (committed ncu summary, source file whose hash the summary records)
TRAFFIC_FILES = {"gemv_t": ("gemv_traffic.txt", "gemv.cuh"), "gemv_n": ("gemv_traffic.txt", "gemv.cuh"),
                 "llt": ("llt_traffic.txt", "llt.cuh"), "llt_tn": ("llt_traffic.txt", "llt.cuh"),
                 "sigma_gemm": ("sigma_traffic.txt", "sigma.cu"),
                 "cs_tn": ("countsketch_traffic.txt", "countsketch.cu"), "sketch": ("sketch_traffic.txt", "gemm_chunk.cuh")}


def committed_traffic(kernel, layout="nt"):
    """Per-launch DRAM bytes from the committed ncu summary, if it matches this source.

    Entries are keyed by kernel, with a ``_tn`` suffix for the transposed layout."""
    if kernel not in TRAFFIC_FILES:
        return None
    key = kernel if kernel.endswith("_tn") or layout != "tn" else kernel + "_tn"
    fname, srcname = TRAFFIC_FILES[kernel]
    path = os.path.join(ROOT, "profiles", fname)
    if not os.path.exists(path):
        return None
    import hashlib
    src = os.path.join(ROOT, "paper_2604_02917_gb300", "csrc", srcname)
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    vals = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha", vals.get("gemv_source_sha")) != sha:
        return None
    v = vals.get(f"{key}_dram_bytes_per_launch")
    return float(v) if v else None


def roofline(infos, model, dtype, layout="nt"):
    """HBM roofline of the solve loop's dominant L pass from the per-launch CUDA events.

    Algorithmic bytes per launch: the factor once (n T e) plus the vectors the
    pass must read and write (FP8 adds the n row scales)."""
    es = {"f32": 4, "bf16": 2, "fp8": 1}[dtype]
    n, T = model.n, model.T
    nT = n * T
    sc = 4 * n if dtype == "fp8" else 0
    pairs = max(sum(i["timed_pairs"] for i in infos), 1)
    step_us = round(sum(i["t_step_ms"] for i in infos) / pairs * 1e3, 2)
    if all(i.get("fused", 0) for i in infos):
        kern = "llt_tn" if layout == "tn" else "llt"
        avg_ms = sum(i["t_fused_ms"] for i in infos) / pairs
        alg = nT * es + 4 * n + 8 * n + sc          # L, y (FP32), g (FP64)
        other = None
    else:
        tt = sum(i["t_gemv_t_ms"] for i in infos)
        tn = sum(i["t_gemv_n_ms"] for i in infos)
        kern = "gemv_t" if tt >= tn else "gemv_n"
        avg_ms = (tt if kern == "gemv_t" else tn) / pairs
        if kern == "gemv_t":
            alg = nT * es + 4 * n + 4 * T + sc
        else:
            alg = nT * es + 4 * T + 8 * n + sc
        other = round(((tn if kern == "gemv_t" else tt) / pairs) * 1e3, 2)
    achieved = alg / (avg_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": committed_traffic(kern, layout), "kernel": kern,
            "peak_source": peak_kind, "avg_launch_us": round(avg_ms * 1e3, 2),
            "alg_bytes_per_launch": alg, "step_kernel_avg_us": step_us}
    if other is not None:
        roof["other_kernel_avg_us"] = other
    return roof


CLOCK_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")


def parse_clock_samples(lines, t0=None, t1=None, margin=0.1):
    """Summarise nvidia-smi lines (timestamp, index, clocks.sm, clocks.max.sm,
    power.draw, active mask, then the four reasons of CLOCK_REASONS): the
    samples stamped within [t0 - margin, t1 + margin] (host epoch seconds),
    or all of them when none is."""
    rows = []
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 10:
            continue
        try:
            ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            ts = None
        try:
            sm, mx = float(parts[2]), float(parts[3])
        except ValueError:
            continue
        act = {nm for nm, val in zip(CLOCK_REASONS, parts[6:10]) if val.lower().startswith("active")}
        rows.append((ts, sm, mx, act))
    if not rows:
        return None
    window = "timed region"
    keep = [r for r in rows if t0 is not None and t1 is not None and r[0] is not None
            and t0 - margin <= r[0] <= t1 + margin]
    if not keep:
        keep, window = rows, "whole sampling (no sample inside the timed region)"
    reasons = set().union(*(r[3] for r in keep))
    return {"sm_mhz": float(np.median([r[1] for r in keep])), "sm_max_mhz": float(max(r[2] for r in keep)),
            "reasons": sorted(reasons), "samples": len(keep), "window": window}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons around the timed
    region: sampling starts before the warm-up (every 50 ms), ``mark()``
    notes the host time at which the timed region starts, and ``stop()``
    keeps the samples stamped between then and its own call."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_index, period_ms=50):
        self.t0 = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-i", str(dev_index), "-lms", str(period_ms)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def mark(self):
        self.t0 = time.time()

    def stop(self):
        t1 = time.time()
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        out = parse_clock_samples(self.f.read().strip().splitlines(), self.t0, t1)
        os.unlink(self.f.name)
        return out


def oracle_problem(model, R32=None):
    """The FP64 oracle's inputs for the headline workload: mu and L from its
    own centering of the same FP32-rounded panel, the return target and the
    power-method start."""
    from synth import factor_returns, power_start
    from oracle.center import center_factor
    if R32 is None:
        R32 = factor_returns(model, np.float32)
    mu, L, _ = center_factor(R32.astype(np.float64))
    return mu, L, float(np.percentile(mu, 60)), power_start(model.n)


def oracle_solve(mu, L, Rt, r0, eps, power_iters=50, lanczos=0):
    """One complete FP64 oracle solve, timed: the step estimate (the power
    method, or Lanczos steps with ``lanczos=1``), Algorithm 1 with the literal
    KKT test every 5 iterations until the residual is <= eps, and the
    objective (the work of one GPU step; the centering, like the GPU's, is
    outside the timed region)."""
    from oracle.npga import initial_point, lanczos_norm2, npga, power_norm2, step_size
    t0 = time.perf_counter()
    lam = lanczos_norm2(L, r0, power_iters) if lanczos else power_norm2(L, r0, power_iters)
    res = npga(L, 0.0, mu, Rt, initial_point(mu, Rt), step_size(lam, 0.0), eps=eps, max_iter=100000, kkt_every=5)
    return time.perf_counter() - t0, res


def cpu_baseline(model, eps, R32=None, x_gpu=None, f_gpu=None, prob=None, sopts=None, slabel="50 power iterations"):
    """The FP64 oracle on this host's cores: one complete solve of the
    headline workload (not a sample), with its own iteration count and its
    distance to the GPU's answer."""
    mu, L, Rt, r0 = oracle_problem(model, R32) if prob is None else prob
    t, res = oracle_solve(mu, L, Rt, r0, eps, **(sopts or {}))
    out = {"value": t, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": f"full solve: FP64 NumPy oracle on the whole {model.n}x{model.T} matrix, {slabel} "
                     f"+ Algorithm 1 with the literal KKT test every 5 iterations to {eps:g} "
                     f"({res.iters} iterations, KKT {res.kkt:.2e}) + objective",
           "iterations": res.iters, "kkt": res.kkt, "objective": res.f}
    if x_gpu is not None:
        out["x_inf_vs_gpu"] = float(np.max(np.abs(np.asarray(x_gpu) - res.x)))
    if f_gpu is not None:
        out["rel_obj_gpu_vs_oracle"] = (f_gpu - res.f) / res.f
    return out


def row_oracles(model, R32, res, prob=None, sopts=None):
    """The FP64 oracle timed beside each further row, on the host cores, as it
    stands.  Each row runs the whole workload where that takes well under a
    minute (the sketch, the CountSketch, the truncation, the explicit-Sigma
    formation and solve, the 64-target frontier at 200 x 1000, the adjoint);
    the frontier at the full shape and the uneven batch would take several
    minutes, so they are timed on a stated sample and scaled (marked
    "scaled": true)."""
    from synth import CFG_SMALL, countsketch_hash, gaussian_sketch, power_start
    from oracle.center import center_factor
    from oracle.npga import (gradient, initial_point, lanczos_norm2, npga, npga_sigma, power_norm2,
                             power_norm2_sigma, sigma_from_factor, step_size)
    from oracle.projection import project_F
    from oracle import adjoint as oadj
    from oracle import strmodel
    cores = os.cpu_count()
    out = {}
    n, T, m = model.n, model.T, 8192
    sopts = sopts or {"power_iters": 50}

    def lam_est(Lx, rx):
        """The step estimate the GPU rows use (Lanczos steps or power iterations)."""
        if sopts.get("lanczos", 0):
            return lanczos_norm2(Lx, rx, sopts["power_iters"])
        return power_norm2(Lx, rx, sopts["power_iters"])

    def full(t, sample):
        return {"value": t, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample, "scaled": False}

    def scaled(t_sample, scale, sample):
        return {"value": t_sample * scale, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample,
                "sample_s": round(t_sample, 3), "scale": round(scale, 2), "scaled": True}

    mu, L, Rt, r0 = oracle_problem(model, R32) if prob is None else prob
    # a8 Gaussian sketch L Phi, whole product
    Phi_t = gaussian_sketch(T, m, seed=2)
    t0 = time.perf_counter()
    Lt = strmodel.sketch(L, Phi_t)
    out["sketch"] = full(time.perf_counter() - t0, f"the whole L Phi: {n} x {T} times {T} x {m} in FP64")
    del Phi_t
    # a9 truncation of that sketch: K = tilde L tilde L^T and eigh (all n pairs), top 512 kept
    t0 = time.perf_counter()
    strmodel.truncate(Lt, 512)
    out["truncate"] = full(time.perf_counter() - t0, f"K = tilde L tilde L^T ({n} x {n}) and eigh, k = 512")
    del Lt
    # f2 CountSketch (dense Phi, as the oracle states it), whole product
    h, sg = countsketch_hash(T, m, seed=2)
    t0 = time.perf_counter()
    strmodel.countsketch(L, h, sg, m)
    out["countsketch"] = full(time.perf_counter() - t0, f"the whole L Phi with the dense {T} x {m} CountSketch Phi")
    # f1 explicit Sigma: formation + the whole solve (50 power iterations on Sigma + Algorithm 1 to 1e-6)
    t0 = time.perf_counter()
    Sig = sigma_from_factor(L)
    t_form = time.perf_counter() - t0
    t0 = time.perf_counter()
    rs_ = npga_sigma(Sig, 0.0, mu, Rt, initial_point(mu, Rt), step_size(power_norm2_sigma(Sig, r0, 50), 0.0),
                     eps=1e-6, max_iter=100000)
    t_solve = time.perf_counter() - t0
    out["sigma"] = dict(full(t_form + t_solve, f"Sigma = L L^T in FP64 ({t_form:.1f} s) + the whole solve on it "
                                               f"({t_solve:.2f} s, {rs_.iters} iterations)"),
                        form_s=t_form, solve_s=t_solve)
    del Sig
    # a11 frontier at 200 x 1000: all 64 targets, each a full solve
    Rf = factor_returns_small()
    muf, Lf, _ = center_factor(Rf)
    tg = np.linspace(np.percentile(muf, 10), np.percentile(muf, 90), 64)
    t0 = time.perf_counter()
    lam = lam_est(Lf, power_start(Lf.shape[0]))
    for r in tg:
        npga(Lf, 0.0, muf, float(r), initial_point(muf, float(r)), step_size(lam, 0.0), eps=1e-6, max_iter=20000)
    out["frontier_200x1000"] = full(time.perf_counter() - t0, "all 64 targets at 200 x 1000, each solved to 1e-6")
    # a11 frontier at the full shape: 2 of the 64 targets solved in full, scaled by 32
    tgf = np.linspace(np.percentile(mu, 10), np.percentile(mu, 90), 64)
    t0 = time.perf_counter()
    lamf = lam_est(L, r0)
    for r in (tgf[0], tgf[63]):
        npga(L, 0.0, mu, float(r), initial_point(mu, float(r)), step_size(lamf, 0.0), eps=1e-6, max_iter=100000)
    out["frontier_full_shape"] = scaled(time.perf_counter() - t0, 32.0,
                                        "targets 1 and 64 of 64 at the full shape, each a full solve, scaled by 32")
    # plain NPGA at 200 x 1000: the whole 2000-iteration run, and the GPU's x against it
    if res.get("small_x") is not None:
        Rt1 = float(np.percentile(muf, 60))
        t0 = time.perf_counter()
        lam1 = power_norm2(Lf, power_start(Lf.shape[0]), 50)
        ref = npga(Lf, 0.0, muf, Rt1, initial_point(muf, Rt1), step_size(lam1, 0.0), eps=0.0, max_iter=2000)
        t1 = time.perf_counter() - t0
        xg = np.asarray(res["small_x"], dtype=np.float64)
        fo = float(np.sum((Lf.T @ ref.x) ** 2))
        fg = float(np.sum((Lf.T @ xg) ** 2))
        out["small_200x1000"] = dict(full(t1, "the whole solve: 50 power + 2000 NPGA iterations"),
                                     x_inf_err=float(np.max(np.abs(xg - ref.x))), rel_obj_err=(fg - fo) / fo)
    # a13 adjoint: the whole 500-iteration forward (with its tape) and reverse sweep at 2000 x 10000
    am = CFG_SMALL.scaled(2000, 10000, seed=0)
    from synth import factor_returns
    mua, La, _ = center_factor(factor_returns(am, np.float32).astype(np.float64))
    Rta = float(np.percentile(mua, 60))
    x0 = initial_point(mua, Rta)
    a = step_size(power_norm2(La, power_start(am.n), 50), 0.0)
    t0 = time.perf_counter()
    x, tape, betas = oadj.unrolled_forward(La, 0.0, mua, Rta, x0, a, 500, record=True)
    t_f = time.perf_counter() - t0
    oadj.backward(La, 0.0, mua, a, tape, betas, np.ones(am.n))
    t_all = time.perf_counter() - t0
    out["adjoint"] = dict(full(t_all, f"forward ({t_f:.1f} s) + reverse of all 500 iterations at 2000 x 10000"),
                          forward_s=t_f, backward_s=t_all - t_f)
    del tape
    # a12 batch: the oracle's per-iteration cost is proportional to n T; time 3 iterations at 1000 x 4000
    # and scale by the batch's sum over problems of n_j T_j (50 power + its iterations)
    if res.get("batch_elem_iters"):
        Lb = La[:1000, :4000]
        mub = mua[:1000]
        Rtb = float(np.percentile(mub, 60))
        yb = initial_point(mub, Rtb)
        t0 = time.perf_counter()
        for _ in range(3):
            project_F(yb - 1e-3 * gradient(Lb, 0.0, yb), mub, Rtb)
        t_el = (time.perf_counter() - t0) / 3 / (1000 * 4000)
        out["batch"] = scaled(t_el * 1000 * 4000, res["batch_elem_iters"] / (1000 * 4000),
                              "3 iterations at 1000 x 4000, scaled by sum_j n_j T_j (50 + iterations_j)")
    return out


def factor_returns_small():
    from synth import CFG_SMALL, factor_returns
    return factor_returns(CFG_SMALL, np.float32).astype(np.float64)


def reference_arm(args):
    """The reference arm: the FP64 oracle (the CPU restatement of the method)
    on the host cores, each step one complete solve of the same workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    model = workload(args, 0)
    prob = oracle_problem(model)
    sopts, slabel = step_opts(args)
    vals = []
    res = None
    for i in range(args.warmup + args.steps):
        t, res = oracle_solve(*prob, args.eps, **sopts)
        if i >= args.warmup:
            vals.append(t)
    v = float(np.mean(vals))
    cb = {"value": v, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
          "sample": f"each step one full solve: {slabel} + Algorithm 1 with the literal KKT test every 5 "
                    f"iterations to {args.eps:g} ({res.iters} iterations) on the whole {model.n}x{model.T} matrix",
          "iterations": res.iters, "kkt": res.kkt}
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"npga full model n={model.n} T={model.T}, FP64 oracle, step from {slabel}",
                       "n": model.n, "T": model.T, "kkt_eps": args.eps, "step_estimate": slabel},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profile_run(args):
    """One instance of a workload for a profiler: the sketch GEMM (L in BF16
    times a Phi drawn from seed 2, m = --sketch-m), one 64-target frontier
    solve (BF16, or FP8 with --dtype fp8; targets between the 10th and 90th
    percentiles of mu), or
    one solve of the first --batch-count problems of the uneven batch (FP32,
    L stored transposed; a warm-up solve first), or one STR build from the
    seed (mv_sketch_str: draw, sketch, truncation to --str-k; a warm-up build
    first), or one reverse sweep of 500 unrolled iterations at 2000 x 10000
    (checkpoints every 50; a warm-up sweep first)."""
    import torch
    from paper_2604_02917_gb300 import mv
    from synth import factor_returns
    if args.profile == "adjoint":
        from synth import CFG_SMALL
        am = CFG_SMALL.scaled(2000, 10000, seed=0)
        La, _, mua, _ = mv.center_factor(torch.from_numpy(factor_returns(am, np.float32)).cuda(), "f32")
        Rta = float(np.percentile(mua.cpu().numpy(), 60))
        g = torch.randn(am.n, dtype=torch.float64, device="cuda",
                        generator=torch.Generator(device="cuda").manual_seed(0))
        mv.npga_backward(La, mua, Rta, am.T, g, 500, checkpoint_every=50)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mv.npga_backward(La, mua, Rta, am.T, g, 500, checkpoint_every=50)
        e1.record()
        torch.cuda.synchronize()
        print(f"adjoint 2000x10000, 500 iterations: backward {e0.elapsed_time(e1):.3f} ms", flush=True)
        return
    if args.profile == "batch":
        from synth import factor_returns_device, uneven_problem_sizes
        probs = []
        for bm in uneven_problem_sizes(args.batch_count):
            Rb = factor_returns_device(bm, torch.device("cuda"))
            Lb, _, mub, _ = mv.center_factor(Rb, "f32", layout="tn")
            del Rb
            probs.append({"L": Lb, "mu": mub, "R_target": float(torch.quantile(mub, 0.6).item()), "T": bm.T,
                          "layout": "tn"})
        bsv = mv.BatchSolver(probs, eps=args.eps)
        bsv.solve()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, infos = bsv.solve()
        e1.record()
        torch.cuda.synchronize()
        its = sorted(i["iterations"] for i in infos)
        print(f"batch {len(probs)} problems: {e0.elapsed_time(e1):.3f} ms; iterations " + " ".join(map(str, its)),
              flush=True)
        return
    model = workload(args, 0)
    R = torch.from_numpy(factor_returns(model, np.float32)).cuda()
    low = "fp8" if (args.profile == "frontier" and args.dtype == "fp8") else "bf16"
    L, rs, mu, _ = mv.center_factor(R, low)
    del R
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.profile == "sketch":
        Phi = mv.gaussian_sketch(2, args.sketch_m, model.T)
        e0.record()
        mv.sketch(L, model.T, Phi)
        e1.record()
    elif args.profile == "str":
        mv.sketch_str(L, model.T, args.sketch_m, 2, args.str_k, "bf16")
        torch.cuda.synchronize()
        e0.record()
        mv.sketch_str(L, model.T, args.sketch_m, 2, args.str_k, "bf16")
        e1.record()
    else:
        muh = mu.cpu().numpy()
        tg = np.linspace(np.percentile(muh, 10), np.percentile(muh, 90), 64)
        fs = mv.FrontierSolver(L, mu, tg, model.T, eps=args.eps, dtype=low, row_scale=rs)
        e0.record()
        fs.solve()
        e1.record()
    torch.cuda.synchronize()
    print(f"{args.profile} {model.n}x{model.T}: {e0.elapsed_time(e1):.3f} ms", flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.profile:
        return profile_run(args)
    import torch
    from paper_2604_02917_gb300 import mv
    from synth import factor_returns, power_start

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    model = workload(args, rank)
    R32 = factor_returns(model, np.float32)
    R_dev = torch.from_numpy(R32).to(dev)
    L, rs, mu, tr = mv.center_factor(R_dev, args.dtype, layout=args.layout)
    Rt = float(np.percentile(mu.cpu().numpy(), 60))
    r0 = torch.from_numpy(power_start(model.n)).to(dev)
    sopts, slabel = step_opts(args)
    # The timed solves replay each chunk of kkt_every iterations as one CUDA
    # graph (the product path); a separate solve issues every launch from the
    # host between CUDA events for the per-kernel breakdown and the roofline.
    solver = mv.Solver(L, mu, Rt, model.T, dtype=args.dtype, row_scale=rs, power_start=r0, eps=args.eps,
                       layout=args.layout, two_pass=1 if args.two_pass else 0, **sopts)
    del R_dev

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def launch_profile(*a, **kw):
        sv = mv.Solver(*a, timing=1, **kw)
        sv.solve()
        out = [sv.solve()[1] for _ in range(2)]
        del sv
        return out

    clk = Clocks(local)
    for _ in range(args.warmup):
        solver.solve()
    barrier()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    barrier()
    clk.mark()
    ev0.record(stream)
    for _ in range(args.steps):
        _, info = solver.solve()
        infos.append(info)
    ev1.record(stream)
    barrier()
    clocks = clk.stop()
    x_head = solver.x.cpu().numpy()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world, dev)
    tinfos = launch_profile(L, mu, Rt, model.T, dtype=args.dtype, row_scale=rs, power_start=r0, eps=args.eps,
                            layout=args.layout, two_pass=1 if args.two_pass else 0, **sopts)

    # roofline of the dominant kernel (per-launch CUDA events around every loop launch)
    roof = roofline(tinfos, model, args.dtype, args.layout)
    es = {"f32": 4, "bf16": 2, "fp8": 1}[args.dtype]
    nT = model.n * model.T

    # end to end through host buffers: upload R, center, solve, download x
    e2e = None
    if not args.no_e2e:
        R_pin = torch.from_numpy(R32).pin_memory()
        x_host = torch.empty(model.n, dtype=torch.float64).pin_memory()
        cws = torch.empty(mv.lib().mv_center_host_workspace_size(model.n, model.T), dtype=torch.uint8, device=dev)
        e_solver = None
        e_times, e_up = [], []
        for i in range(2 + 3):
            torch.cuda.synchronize()
            a0 = torch.cuda.Event(enable_timing=True)
            am = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            # upload of R overlapped with its centering, chunk by chunk (mv_center_factor_host)
            L2, rs2, mu2, _ = mv.center_factor_host(R_pin, args.dtype, layout=args.layout, device=dev, ws=cws)
            am.record(stream)
            if e_solver is None:
                e_solver = mv.Solver(L2, mu2, Rt, model.T, dtype=args.dtype, row_scale=rs2, power_start=r0,
                                     eps=args.eps, layout=args.layout, **sopts)
            else:
                e_solver.problem.L = L2.data_ptr()
                e_solver.problem.mu = mu2.data_ptr()
                e_solver.problem.row_scale = None if rs2 is None else rs2.data_ptr()
                e_solver._keep = (L2, mu2, rs2, r0)
            x, _ = e_solver.solve()
            x_host.copy_(x, non_blocking=True)
            a1.record(stream)
            torch.cuda.synchronize()
            if i >= 2:
                e_times.append(a0.elapsed_time(a1))
                e_up.append(a0.elapsed_time(am))
            # release this step's factor before the next upload: the next one
            # reuses the same device block (and the solver's cached graph)
            e_solver._keep = None
            del L2, mu2, rs2
        e2e = {"value": float(np.mean(e_times)) / 1e3, "unit": "s",
               "h2d_bytes_per_step": int(R32.nbytes), "d2h_bytes_per_step": int(model.n * 8),
               "upload_center_s": float(np.mean(e_up)) / 1e3,
               "upload_GBps": R32.nbytes / (float(np.mean(e_up)) / 1e3) / 1e9}
        del R_pin, cws

    # Low-precision storage + FP32 refinement on the same workload and GPU.
    variants = {}

    def timed_solves(sv):
        for _ in range(args.warmup):
            sv.solve()
        torch.cuda.synchronize()
        v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        vinfos = []
        v0.record(stream)
        for _ in range(args.steps):
            _, vi = sv.solve()
            vinfos.append(vi)
        v1.record(stream)
        torch.cuda.synchronize()
        return v0.elapsed_time(v1) / args.steps / 1e3, vinfos

    if not args.no_variants:
        # The same FP32 solve with the two half-products as separate passes, and
        # in the other layout: the path from two passes over n x T to one pass
        # over L^T.
        R_dev = torch.from_numpy(R32).to(dev)
        other = "nt" if args.layout == "tn" else "tn"
        Lo, rso, _, _ = mv.center_factor(R_dev, args.dtype, layout=other)
        del R_dev
        for name, LL, rr, lay, two in ((f"{args.dtype}_{args.layout}_two_pass", L, rs, args.layout, 1),
                                       (f"{args.dtype}_{other}_fused", Lo, rso, other, 0),
                                       (f"{args.dtype}_{other}_two_pass", Lo, rso, other, 1)):
            kw = dict(dtype=args.dtype, row_scale=rr, power_start=r0, eps=args.eps, two_pass=two, layout=lay, **sopts)
            sv = mv.Solver(LL, mu, Rt, model.T, **kw)
            t, vinfos = timed_solves(sv)
            pinfos = launch_profile(LL, mu, Rt, model.T, **kw)
            variants[name] = {"value": t, "unit": "s", "iterations": vinfos[-1]["iterations"],
                              "kkt": vinfos[-1]["kkt"], "objective": vinfos[-1]["objective"],
                              "fused": vinfos[-1]["fused"], "roofline": roofline(pinfos, model, args.dtype, lay)}
            del sv
        del Lo, rso
        # The headline solve with the power method of the Sec. 3.1 remark for
        # lambda_hat: 50 iterations, and 10 (the remark's "a handful").
        for it in (50, 10):
            kw = dict(dtype=args.dtype, row_scale=rs, power_start=r0, eps=args.eps, layout=args.layout,
                      two_pass=1 if args.two_pass else 0, power_iters=it)
            sv = mv.Solver(L, mu, Rt, model.T, **kw)
            t, vinfos = timed_solves(sv)
            vi = vinfos[-1]
            variants[f"{args.dtype}_{args.layout}_power{it}"] = {
                "value": t, "unit": "s", "power_iters": it, "iterations": vi["iterations"], "kkt": vi["kkt"],
                "converged": vi["converged"], "objective": vi["objective"], "lambda_hat": vi["lambda_hat"],
                "lambda_hat_over_headline": vi["lambda_hat"] / infos[-1]["lambda_hat"],
                "rel_obj_vs_headline": (vi["objective"] - infos[-1]["objective"]) / infos[-1]["objective"]}
            del sv
    if not args.no_variants and args.dtype == "f32":
        R_dev = torch.from_numpy(R32).to(dev)
        for vdt in ("bf16", "fp8"):
            # low-precision copy n x T (its faster layout), FP32 refinement on the headline L
            Llo, rslo, _, _ = mv.center_factor(R_dev, vdt, layout="nt")
            rsv = mv.RefinedSolver(Llo, L, mu, Rt, model.T, dtype=vdt, row_scale=rslo, power_start=r0,
                                   eps_lo=1e-5, eps=args.eps, layout="nt", layout_hi=args.layout, **sopts)
            for _ in range(args.warmup):
                rsv.solve()
            torch.cuda.synchronize()
            v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            v0.record(stream)
            for _ in range(args.steps):
                _, vi = rsv.solve()
            v1.record(stream)
            torch.cuda.synchronize()
            variants[vdt + "+fp32_refine"] = {
                "value": v0.elapsed_time(v1) / args.steps / 1e3, "unit": "s", "iterations": vi["iterations"],
                "refine_iterations": vi["refine_iterations"], "kkt": vi["kkt"], "objective": vi["objective"],
                "rel_obj_vs_fp32": (vi["objective"] - infos[-1]["objective"]) / infos[-1]["objective"]}
            del Llo, rslo, rsv
        del R_dev

    # Explicit covariance (Sec. 3 remark): Sigma = L L^T once on tcgen05, then
    # NPGA with one symmetric pass over the upper triangle of Sigma per iteration.
    sigma_res = None
    if not args.no_sigma and args.dtype == "f32":
        R_dev = torch.from_numpy(R32).to(dev)
        sigma_res = {}
        peak_tf, peak_tf_src = peaks_tensor()
        for sdt in ("f32", "bf16"):
            Lx, rsx, _, _ = mv.center_factor(R_dev, sdt, layout="nt")
            S = mv.sigma_form(Lx, model.T, sdt, rsx)              # warm-up (attributes, tensor maps)
            ft = []
            for _ in range(3):
                f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                f0.record(stream)
                S = mv.sigma_form(Lx, model.T, sdt, rsx)
                f1.record(stream)
                torch.cuda.synchronize()
                ft.append(f0.elapsed_time(f1) / 1e3)
            t_form = float(np.median(ft))
            nb = -(-model.n // 128)
            segs = 3 if sdt == "f32" else 1
            flops = nb * (nb + 1) // 2 * 128 * 128 * (-(-model.T // 64) * 64) * 2 * segs
            entry = {"form_s": t_form,
                     "form_roofline": {"bound": "tensor", "achieved": round(flops / t_form / 1e12, 1),
                                       "peak": peak_tf, "peak_source": peak_tf_src, "unit": "TFLOP/s",
                                       "frac": round(flops / t_form / 1e12 / peak_tf, 4),
                                       "traffic": committed_traffic("sigma_gemm") if sdt == "f32" and
                                       (model.n, model.T) == (5440, 48374) else None,
                                       "kernel": "sigma_gemm", "flops_per_launch": flops,
                                       "note": "executed BF16 tile flops (upper tiles x segments)"}}
            sv = mv.Solver(S, mu, Rt, model.T, power_start=r0, eps=args.eps, layout="sigma")
            t_solve, vinfos = timed_solves(sv)
            pinfos = launch_profile(S, mu, Rt, model.T, power_start=r0, eps=args.eps, layout="sigma")
            pairs = max(sum(i["timed_pairs"] for i in pinfos), 1)
            symv_us = sum(i["t_fused_ms"] for i in pinfos) / pairs * 1e3
            tri = model.n * (model.n + 1) // 2 * 4
            entry.update({"solve_s": t_solve, "total_s": t_form + t_solve,
                          "iterations": vinfos[-1]["iterations"], "kkt": vinfos[-1]["kkt"],
                          "objective": vinfos[-1]["objective"],
                          "rel_obj_vs_factor_solve": (vinfos[-1]["objective"] - infos[-1]["objective"])
                          / infos[-1]["objective"],
                          "symv": {"avg_launch_us": round(symv_us, 2), "tri_bytes": tri,
                                   "GBps": round(tri / (symv_us * 1e-6) / 1e9, 1),
                                   "note": "upper triangle of Sigma per launch; event-timed host-issued "
                                           "launches (includes enqueue gaps; the ncu launch list has "
                                           "device durations)"},
                          "step_kernel_avg_us": round(sum(i["t_step_ms"] for i in pinfos) / pairs * 1e3, 2)})
            sigma_res[sdt + "_L"] = entry
            del sv, S, Lx, rsx
        del R_dev
        torch.cuda.empty_cache()

    # Sketch (tcgen05 BF16 GEMM) + FP64 truncation + NPGA on the STR model.
    str_res = None
    # the committed ncu traffic of the sketch and CountSketch kernels was taken at this shape
    full_cs_shape = (model.n, model.T, args.sketch_m) == (5440, 48374, 8192)
    if not args.no_str and args.dtype == "f32":
        R_dev = torch.from_numpy(R32).to(dev)
        Lb, _, _, trd = mv.center_factor(R_dev, "bf16")
        del R_dev
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

        def timed(fn, reps=3):
            fn()                                                   # warm-up (attributes, tensor maps, libraries)
            ts = []
            for _ in range(reps):
                e[0].record(stream)
                out = fn()
                e[1].record(stream)
                torch.cuda.synchronize()
                ts.append(e[0].elapsed_time(e[1]))
            return min(ts), out

        # the stages one by one: Phi drawn from the seed on the device, the sketch GEMM, the truncation
        gen_ms, Phi_t = timed(lambda: mv.gaussian_sketch(2, args.sketch_m, model.T))
        sk_ms, Ls = timed(lambda: mv.sketch(Lb, model.T, Phi_t))
        flop = 2.0 * model.n * model.T * args.sketch_m
        t_first = time.perf_counter()
        mv.str_truncate(Ls, args.str_k, -1.0, float(trd.cpu()))
        t_first = time.perf_counter() - t_first
        tr_ms, _ = timed(lambda: mv.str_truncate(Ls, args.str_k, -1.0, float(trd.cpu())))
        # the whole STR build through its one call (seed in, L_eff out)
        build_ms, (L_eff, sigma, gamma, _) = timed(
            lambda: mv.sketch_str(Lb, model.T, args.sketch_m, 2, args.str_k, "bf16", None, -1.0, float(trd.cpu()),
                                  keep_sketch=False))
        sk_ms = [sk_ms]
        # kappa(hat Sigma) ~ 4e4: a 1e-6 KKT residual leaves the objective ~2e-3 above the STR optimum
        # (1e-8: 3e-5), so the STR model is solved to 1e-9 (x within 1e-4 of the oracle's, objective 1e-5)
        str_eps = min(args.eps, 1e-9)
        ssv = mv.Solver(L_eff, mu, Rt, args.str_k, gamma=gamma, power_start=r0, eps=str_eps, **sopts)
        for _ in range(args.warmup):
            ssv.solve()
        torch.cuda.synchronize()
        e[0].record(stream)
        for _ in range(args.steps):
            xs, si = ssv.solve()
        e[1].record(stream)
        torch.cuda.synchronize()
        s_ms = e[0].elapsed_time(e[1]) / args.steps
        # the same solve to the headline's KKT tolerance
        ssv6 = mv.Solver(L_eff, mu, Rt, args.str_k, gamma=gamma, power_start=r0, eps=args.eps, **sopts)
        for _ in range(args.warmup):
            ssv6.solve()
        torch.cuda.synchronize()
        e[0].record(stream)
        for _ in range(args.steps):
            _, si6 = ssv6.solve()
        e[1].record(stream)
        torch.cuda.synchronize()
        s6_ms = e[0].elapsed_time(e[1]) / args.steps
        del ssv6
        _, gfull = mv.gradient(L, xs, model.T, layout=args.layout, with_z=False)  # 2 L L^T x, full FP32 model
        f_str_full = float(torch.dot(xs, gfull).item()) / 2.0
        f_full = infos[-1]["objective"]
        bf16_peak, bf16_src = peaks_tensor()
        tflops = flop / (min(sk_ms) * 1e-3) / 1e12
        str_res = {"gaussian_draw": {"ms": gen_ms, "entries": args.sketch_m * model.T, "seed": 2,
                                     "note": "Phi^T drawn on the device (Philox4x32-10 + Box-Muller, BF16)"},
                   "sketch": {"m": args.sketch_m, "ms": min(sk_ms), "tflop": flop / 1e12,
                              "achieved_tflops": round(tflops, 1), "peak_tflops": bf16_peak, "peak_source": bf16_src,
                              "frac": round(tflops / bf16_peak, 4), "bound": "tensor",
                              "traffic": committed_traffic("sketch") if full_cs_shape else None},
                   "truncate": {"k": args.str_k, "ms": tr_ms, "first_call_s": round(t_first, 3), "gamma": gamma,
                                "sigma_1": float(sigma[0]),
                                "sigma_k": float(sigma[-1])},
                   "solve": {"value": s_ms / 1e3, "unit": "s", "iterations": si["iterations"], "kkt": si["kkt"],
                             "kkt_eps": str_eps, "step_estimate": slabel},
                   "solve_headline_eps": {"value": s6_ms / 1e3, "unit": "s", "iterations": si6["iterations"],
                                          "kkt": si6["kkt"], "kkt_eps": args.eps},
                   "full_model_gap": (f_str_full - f_full) / f_full,
                   "build_ms": build_ms,
                   "build_plus_solve_s": (build_ms + s_ms) / 1e3,
                   "note": "build = mv_sketch_str: Phi drawn from the seed + sketch + truncation, one call"}
        del Lb, Phi_t, Ls, L_eff, ssv
        # CountSketch alternative (Sec. 2.3 (2)) on the headline factor: one HBM pass over L.
        from synth import countsketch_hash
        hh, sg = countsketch_hash(model.T, args.sketch_m, seed=2)
        hh, sg = torch.from_numpy(hh).to(dev), torch.from_numpy(sg).to(dev)
        es_h = {"f32": 4, "bf16": 2, "fp8": 1}[args.dtype]
        mv.countsketch(L, model.n, model.T, hh, sg, args.sketch_m, args.dtype, rs, args.layout)   # warm-up
        cs_ms = []
        for _ in range(3):
            e[0].record(stream)
            Lc = mv.countsketch(L, model.n, model.T, hh, sg, args.sketch_m, args.dtype, rs, args.layout)
            e[1].record(stream)
            torch.cuda.synchronize()
            cs_ms.append(e[0].elapsed_time(e[1]))
        cs_bytes = model.n * model.T * es_h + 5 * model.T + 4 * model.n * args.sketch_m
        peak, peak_kind = peaks()
        cs_gbs = cs_bytes / (min(cs_ms) * 1e-3) / 1e9
        str_res["countsketch"] = {"m": args.sketch_m, "layout": args.layout, "dtype": args.dtype,
                                  "ms": min(cs_ms), "alg_bytes": cs_bytes,
                                  "roofline": {"bound": "hbm", "achieved": round(cs_gbs, 1), "peak": peak,
                                               "unit": "GB/s", "frac": round(cs_gbs / peak, 4),
                                               "peak_source": peak_kind,
                                               "traffic": committed_traffic("cs_tn") if full_cs_shape and
                                               args.layout == "tn" and args.dtype == "f32" else None,
                                               "note": "whole call (bucket lists + gather), event-timed; "
                                                       "traffic: the gather kernel's ncu DRAM bytes"}}
        del Lc, hh, sg

    # Plain NPGA at 200 x 1000 (5 factors, seed 0): 2000 iterations, no early
    # stop; L (800 KB) stays on chip, so this measures per-iteration latency.
    small = None
    if not args.no_small and args.dtype == "f32":
        from synth import CFG_SMALL
        Rs = torch.from_numpy(factor_returns(CFG_SMALL, np.float32)).to(dev)
        Lsm, _, musm, _ = mv.center_factor(Rs, "f32")
        del Rs
        Rts = float(np.percentile(musm.cpu().numpy(), 60))
        r0s = torch.from_numpy(power_start(CFG_SMALL.n)).to(dev)
        ssv = mv.Solver(Lsm, musm, Rts, CFG_SMALL.T, power_start=r0s, eps=0.0, max_iter=2000)
        t, sinfos = timed_solves(ssv)
        xs, _ = ssv.solve()
        small = {"n": CFG_SMALL.n, "T": CFG_SMALL.T, "iterations": sinfos[-1]["iterations"], "value": t, "unit": "s",
                 "us_per_iteration": t / 2000 * 1e6, "kkt": sinfos[-1]["kkt"], "objective": sinfos[-1]["objective"],
                 "note": "whole solve (50 power iterations + 2000 NPGA iterations + objective), KKT test every 5"}
        small_x = xs.cpu().numpy()
        del ssv, Lsm, musm, r0s, xs

    # 64-point efficient frontier (shared BF16 factor, skinny tcgen05 GEMMs).
    frontier = None
    if not args.no_frontier and args.dtype == "f32":
        from synth import CFG_SMALL
        frontier = {}
        for tag, fm, fdt, refine in (("200x1000", CFG_SMALL, "bf16", False), ("full_shape", model, "bf16", False),
                                     ("full_shape_bf16+fp32_refine", model, "bf16", True),
                                     ("200x1000_fp8", CFG_SMALL, "fp8", False), ("full_shape_fp8", model, "fp8", False)):
            Rf = factor_returns(fm, np.float32) if fm is not model else R32
            Rfd = torch.from_numpy(Rf).to(dev)
            Lfb, rsf, muf, _ = mv.center_factor(Rfd, fdt)
            Lhi = mv.center_factor(Rfd, "f32")[0] if refine else None
            muh = muf.cpu().numpy()
            targets = np.linspace(np.percentile(muh, 10), np.percentile(muh, 90), 64)
            fsv = mv.FrontierSolver(Lfb, muf, targets, fm.T, eps=args.eps, dtype=fdt, row_scale=rsf, L_f32=Lhi,
                                    eps_lo=1e-5, **sopts)
            fsv.solve()
            torch.cuda.synchronize()
            reps = 3 if tag.startswith("full_shape") else 5
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for _ in range(reps):
                _, finfo = fsv.solve()
            f1.record(stream)
            torch.cuda.synchronize()
            entry = {"targets": 64, "value": f0.elapsed_time(f1) / reps / 1e3, "unit": "s",
                     "max_iterations": max(i["iterations"] for i in finfo),
                     "all_converged": all(i["converged"] == 1 for i in finfo), "dtype": fdt,
                     "kkt_eps": args.eps, "model": "fp32 (refined)" if refine else fdt, "step_estimate": slabel}
            if refine:
                entry["max_refine_iterations"] = max(i["refine_iterations"] for i in finfo)
                entry["note"] = ("BF16 frontier to KKT 1e-5, then every target refined on the FP32 factor "
                                 "(BF16 hi + lo pair) to the KKT tolerance on the FP32 model")
            # algorithmic bytes: the step estimate's fused passes over L + two GEMMs (L^T and L) per loop iteration
            fe = 2 if fdt == "bf16" else 1
            kp = sopts["power_iters"]
            if refine:       # phase 2 reads both BF16 parts in each GEMM
                it2 = entry["max_refine_iterations"]
                fbytes = fm.n * fm.T * 2 * (kp + 2 * (entry["max_iterations"] - it2 + 1) + 4 * (it2 + 1))
            else:
                fbytes = fm.n * fm.T * fe * (kp + 2 * (entry["max_iterations"] + 1))
            peak, peak_kind = peaks()
            fgbs = fbytes / entry["value"] / 1e9
            entry["roofline"] = {"bound": "hbm", "achieved": round(fgbs, 1), "peak": peak, "unit": "GB/s",
                                 "frac": round(fgbs / peak, 4), "peak_source": peak_kind, "traffic": None,
                                 "note": "L is L2-resident at 200 x 1000" if fm is not model else "algorithmic"}
            if tag == "200x1000":
                # the same 64 targets as independent FP32 solves, one after another
                Lf32, _, _, _ = mv.center_factor(Rfd, "f32")
                t0 = time.perf_counter()
                for r in targets:
                    mv.npga_solve(Lf32, muf, float(r), fm.T, eps=args.eps, **sopts)
                torch.cuda.synchronize()
                entry["fp32_sequential_64_solves_s"] = time.perf_counter() - t0
                del Lf32
            if tag == "full_shape":
                # the same 64 targets as independent FP32 solves of the headline factor, one after another
                # (launches issued from the host: each target would otherwise capture its own graphs)
                ssv = mv.Solver(L, mu, float(targets[0]), model.T, power_start=r0, eps=args.eps, layout=args.layout,
                                two_pass=1 if args.two_pass else 0, use_graph=0, **sopts)
                ssv.solve()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for r in targets:
                    ssv.problem.R_target = float(r)
                    ssv.solve()
                torch.cuda.synchronize()
                entry["fp32_sequential_64_solves_s"] = time.perf_counter() - t0
                del ssv
            frontier[tag] = entry
            del Rfd, Lfb, rsf, fsv, Lhi

    # Adjoint of 500 unrolled iterations at 2000 x 10000 (checkpoints every 50).
    adj = None
    if not args.no_adjoint and args.dtype == "f32":
        from synth import CFG_SMALL
        am = CFG_SMALL.scaled(2000, 10000, seed=0)
        Ra = factor_returns(am, np.float32)
        La, _, mua, _ = mv.center_factor(torch.from_numpy(Ra).to(dev), "f32")
        Rta = float(np.percentile(mua.cpu().numpy(), 60))
        K = 500
        g = torch.randn(am.n, dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(0))
        mv.npga_solve(La, mua, Rta, am.T, eps=0.0, kkt_every=0, max_iter=K)
        mv.npga_backward(La, mua, Rta, am.T, g, K, checkpoint_every=50)
        torch.cuda.synchronize()
        a0, a1, a2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a0.record(stream)
        mv.npga_solve(La, mua, Rta, am.T, eps=0.0, kkt_every=0, max_iter=K)
        a1.record(stream)
        mv.npga_backward(La, mua, Rta, am.T, g, K, checkpoint_every=50)
        a2.record(stream)
        torch.cuda.synchronize()
        fwd, bwd = a0.elapsed_time(a1), a1.elapsed_time(a2)
        adj = {"n": am.n, "T": am.T, "iterations": K, "checkpoint_every": 50, "forward_s": fwd / 1e3,
               "backward_s": bwd / 1e3, "backward_over_forward": bwd / fwd}
        del La, Ra

    # 256 independent problems, n ~ U[500,5000], T ~ U[2000,20000] (grouped launches).
    # Headline: every factor stored transposed, the grouped single pass (L read
    # once per product); beside it the same batch stored n x T on the grouped
    # GEMV pair (L read twice), with the autotuned and the default tiles.
    batch = None
    batch_elem_iters = 0
    if not args.no_batch and args.dtype == "f32":
        from synth import factor_returns_device, uneven_problem_sizes
        models = uneven_problem_sizes(args.batch_count)

        def build(layout):
            probs = []
            for bm in models:
                Rb = factor_returns_device(bm, dev)
                Lb_, _, mub, _ = mv.center_factor(Rb, "f32", layout=layout)
                del Rb
                Rtb = float(torch.quantile(mub, 0.6).item())
                probs.append({"L": Lb_, "mu": mub, "R_target": Rtb, "T": bm.T, "layout": layout})
            return probs

        def timed_batch(bsv):
            b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            b0.record(stream)
            xs_, bi = bsv.solve()
            b1.record(stream)
            torch.cuda.synchronize()
            return b0.elapsed_time(b1) / 1e3, bi, [x.clone() for x in xs_]

        probs = build("tn")
        bsv = mv.BatchSolver(probs, eps=args.eps)
        bsv.solve()
        bt, binfos, bx_tn = timed_batch(bsv)
        del probs, bsv
        torch.cuda.empty_cache()
        probs = build("nt")
        bsv = mv.BatchSolver(probs, eps=args.eps)
        os.environ["MV_BATCH_AUTOTUNE"] = "0"            # the untuned default tiles, for comparison
        bsv.solve()
        bt_default, _, _ = timed_batch(bsv)
        del os.environ["MV_BATCH_AUTOTUNE"]
        bsv.solve()                                      # the first tuned solve times the tile candidates
        torch.cuda.synchronize()
        bt_nt, binfos_nt, bx_nt = timed_batch(bsv)
        t_rows, n_bytes, tuned = bsv.tiles()
        del probs, bsv
        torch.cuda.empty_cache()
        elems = sum(bm.n * bm.T for bm in models)
        iters = [i["iterations"] for i in binfos]
        iters_nt = [i["iterations"] for i in binfos_nt]
        # algorithmic bytes: every L once per product on the transposed layout
        # (50 power steps, the lambda_hat pass, each NPGA iteration, the
        # objective pass); on n x T twice per product and once per z-only pass
        moved = sum(4 * bm.n * bm.T * (50 + 1 + it + 1) for bm, it in zip(models, iters))
        moved_nt = sum(4 * bm.n * bm.T * (2 * 50 + 1 + 2 * it + 1) for bm, it in zip(models, iters_nt))
        batch_elem_iters = sum(bm.n * bm.T * (50 + it + 1) for bm, it in zip(models, iters))
        peak, peak_kind = peaks()
        dx = max(float(torch.max(torch.abs(a - b)).item()) for a, b in zip(bx_tn, bx_nt))
        batch = {"problems": len(models), "elements": elems, "value": bt, "unit": "s", "layout": "tn (grouped single pass)",
                 "roofline": {"bound": "hbm", "achieved": round(moved / bt / 1e9, 1), "peak": peak, "unit": "GB/s",
                              "frac": round(moved / bt / 1e9 / peak, 4), "peak_source": peak_kind, "traffic": None,
                              "note": "one pass of every L per product (algorithmic)"},
                 "problems_per_s": len(models) / bt, "all_converged": all(i["converged"] == 1 for i in binfos),
                 "iterations_min": min(iters), "iterations_max": max(iters),
                 "aggregate_GBps": moved / bt / 1e9, "data": "synthetic, drawn on the GPU (torch seeded stream)",
                 "nt_two_pass": {"value": bt_nt, "unit": "s", "default_tiles_s": bt_default,
                                 "all_converged": all(i["converged"] == 1 for i in binfos_nt),
                                 "roofline_frac": round(moved_nt / bt_nt / 1e9 / peak, 4),
                                 "tiles": {"gemv_t_rows_per_split": t_rows, "gemv_n_bytes_per_split": n_bytes,
                                           "tuned": tuned}},
                 "x_inf_tn_vs_nt": dx}

    cb = None
    if rank == 0 and world == 1 and not args.no_cpu:
        del L
        torch.cuda.empty_cache()
        prob = oracle_problem(model, R32)
        cb = cpu_baseline(model, args.eps, x_gpu=x_head, f_gpu=infos[-1]["objective"], prob=prob,
                          sopts={"lanczos": sopts.get("lanczos", 0), "power_iters": sopts["power_iters"]},
                          slabel=slabel)
        if not args.no_row_oracles:
            res = {"sigma_iters": sigma_res["f32_L"]["iterations"] if sigma_res else 50,
                   "batch_elem_iters": batch_elem_iters, "small_x": small_x if small is not None else None}
            row_cpu = row_oracles(model, R32, res, prob, sopts)
            if str_res is not None:
                for k in ("sketch", "countsketch", "truncate"):
                    if k in str_res:
                        str_res[k]["cpu_oracle"] = row_cpu[k]
            if sigma_res is not None:
                sigma_res["cpu_oracle"] = row_cpu["sigma"]
            if frontier is not None and "200x1000" in frontier:
                frontier["200x1000"]["cpu_oracle"] = row_cpu["frontier_200x1000"]
            if frontier is not None and "full_shape" in frontier:
                frontier["full_shape"]["cpu_oracle"] = row_cpu["frontier_full_shape"]
            if adj is not None:
                adj["cpu_oracle"] = row_cpu["adjoint"]
            if small is not None and "small_200x1000" in row_cpu:
                small["cpu_oracle"] = row_cpu["small_200x1000"]
            if batch is not None and "batch" in row_cpu:
                batch["cpu_oracle"] = row_cpu["batch"]
    if rank == 0:
        last = infos[-1]
        line = {"metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
                "config": {"workload": f"npga full model n={model.n} T={model.T} {args.dtype} L "
                                       f"({'L^T stored T x n' if args.layout == 'tn' else 'n x T'}), "
                                       f"KKT eps={args.eps}, step from {slabel}",
                           "n": model.n, "T": model.T, "kkt_eps": args.eps, "layout": args.layout,
                           "step_estimate": slabel,
                           "l2": "inputs larger than L2 (L is %.2f GB)" % (nT * es / 1e9),
                           "parallelism": "replicas" if world > 1 else "single"},
                "iterations": last["iterations"], "kkt": last["kkt"], "objective": last["objective"],
                "lambda_hat": last["lambda_hat"], "alpha": last["alpha"],
                "gpu_launches": int(sum(i["launches"] for i in infos)),
                "roofline": roof, "cpu_baseline": cb, "e2e": e2e, "clocks": clocks,
                "variants": variants, "sigma": sigma_res, "str": str_res, "small_200x1000": small,
                "frontier": frontier, "adjoint": adj, "batch": batch}
        print(json.dumps(jsonable(line)), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
