"""Multi-rank host logic of bench.py, on the CPU with gloo (world size 2).

Every GPU run here has one GPU, so the N > 1 path is replicas (one
independent problem per rank, weak scaling); what it adds on the host is
checked here: the max-over-ranks time, distinct per-rank workloads, and the
reference arm running on rank 0 only.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = bench.dist_env()
        assert (r, w) == (rank, world)
        m = bench.max_over_ranks(10.0 + 5.0 * rank, world, torch.device("cpu"))
        class A:
            config, shape = "small", None
        wl = bench.workload(A, rank)
        ref = bench.reference_arm(type("B", (), {"gpus": world, "steps": 1, "warmup": 0, "eps": 1e-6,
                                                 "config": "small", "shape": None})) if rank == 1 else None
        out[rank] = (m, wl.seed, wl.n, wl.T, ref)
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    (m0, s0, n0, T0, _), (m1, s1, n1, T1, ref1) = out[0], out[1]
    assert m0 == m1 == 15.0                     # both ranks see the slowest rank's time
    assert s0 != s1 and (n0, T0) == (n1, T1)     # same shape, independent problems (weak scaling)
    assert ref1 is None                          # the reference arm prints on rank 0 only


def test_committed_traffic_lookup(tmp_path, monkeypatch):
    """The bench reports an ncu traffic figure only while the kernel source
    still hashes to the one the summary records."""
    import shutil
    import bench
    for k in bench.TRAFFIC_FILES:
        v = bench.committed_traffic(k, "tn" if k.endswith("_tn") else "nt")
        assert v is None or v > 0
    # a copy of the tree with one source byte changed: no figure
    (tmp_path / "profiles").mkdir()
    (tmp_path / "paper_2604_02917_gb300" / "csrc").mkdir(parents=True)
    shutil.copy(os.path.join(bench.ROOT, "profiles", "countsketch_traffic.txt"), tmp_path / "profiles")
    src = open(os.path.join(bench.ROOT, "paper_2604_02917_gb300", "csrc", "countsketch.cu"), "rb").read()
    (tmp_path / "paper_2604_02917_gb300" / "csrc" / "countsketch.cu").write_bytes(src)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    same = bench.committed_traffic("cs_tn", "tn")
    (tmp_path / "paper_2604_02917_gb300" / "csrc" / "countsketch.cu").write_bytes(src + b"\n")
    assert bench.committed_traffic("cs_tn", "tn") is None
    assert same is None or same > 0


def test_clock_samples_window():
    """Clock samples are summarised over the timed region only (fallback: all)."""
    import datetime
    import bench
    base = datetime.datetime(2026, 1, 2, 3, 4, 5, 0)

    def line(dt_s, sm, pcap="Not Active", hw="Not Active"):
        ts = (base + datetime.timedelta(seconds=dt_s)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"{ts}, 0, {sm}, 2070, 900.5, 0x0, {hw}, Not Active, Not Active, {pcap}"

    lines = [line(0.0, 1200), line(1.0, 2070), line(1.05, 2040, pcap="Active"), line(3.0, 900, hw="Active")]
    t0 = base.timestamp() + 0.95
    out = bench.parse_clock_samples(lines, t0, t0 + 0.2)
    assert out["samples"] == 2 and out["window"] == "timed region"
    assert out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0 and out["reasons"] == ["sw_power_cap"]
    every = bench.parse_clock_samples(lines, t0 + 10.0, t0 + 11.0)
    assert every["samples"] == 4 and every["window"].startswith("whole")
    assert "hw_slowdown" in every["reasons"]
    assert bench.parse_clock_samples(["garbage"], None, None) is None


@pytest.mark.parametrize("est", ["lanczos", "power"])
def test_reference_arm_step_estimate(est, capsys):
    """The reference arm (the FP64 oracle) runs the workload with the step
    estimate the GPU arm uses and labels it; rank 0 prints one JSON line."""
    import json
    import bench
    args = type("B", (), {"gpus": 1, "steps": 1, "warmup": 0, "eps": 1e-6, "config": "small", "shape": None,
                          "step_estimate": est, "step_iters": None})
    sopts, label = bench.step_opts(args)
    assert sopts["power_iters"] == (25 if est == "lanczos" else 50)
    assert sopts.get("lanczos", 0) == (1 if est == "lanczos" else 0)
    bench.reference_arm(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["config"]["step_estimate"] == label
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["kkt"] <= 1e-6
    assert label in line["cpu_baseline"]["sample"]
