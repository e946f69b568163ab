"""The multi-rank path of bench.py on CPU: two gloo ranks, as torchrun would
start them, agree on the slowest rank's time and the whole-job throughput."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    ms_local = [100.0, 130.0][rank]
    ms, value = bench.job_throughput(ms_local, 60, world, torch.device("cpu"))
    dist.barrier()
    out.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == pytest.approx(130.0)
        assert value == pytest.approx(2 * 60 / 0.130)


def test_single_rank_is_local():
    sys.path.insert(0, ROOT)
    import bench
    import torch
    ms, value = bench.job_throughput(80.0, 60, 1, torch.device("cpu"))
    assert ms == 80.0 and value == pytest.approx(60 / 0.080)


def _batch_rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    local = [dict(ms_per_launch=5.0, worst_relres=3e-9, max_its_by_k=[5, 5, 0, 5, 0, 0, 6], iterations=640,
                  outer=0, unknown_iters=1e6, flops=2e9, converged=True),
             dict(ms_per_launch=6.0, worst_relres=9e-9, max_its_by_k=[5, 0, 5, 5, 6, 5, 0], iterations=650,
                  outer=0, unknown_iters=2e6, flops=3e9, converged=False)][rank]
    job = bench.batch_job(local, world, torch.device("cpu"))
    dist.barrier()
    out.put((rank, job))
    dist.destroy_process_group()


def test_two_ranks_combine_the_sharded_batch():
    """The batch section under torchrun: each rank solves its shard; the job
    takes the slowest rank's time, sums the work and converges only if every
    rank did."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batch_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for _, job in res:
        assert job["ms_per_launch"] == pytest.approx(6.0)
        assert job["worst_relres"] == pytest.approx(9e-9)
        assert job["max_its_by_k"] == [5, 5, 5, 5, 6, 5, 6]
        assert job["iterations"] == 1290 and job["outer"] == 0
        assert job["unknown_iters"] == pytest.approx(3e6) and job["flops"] == pytest.approx(5e9)
        assert job["converged"] is False


def test_batch_shards_cover_every_instance_once_and_balance_the_cost():
    sys.path.insert(0, ROOT)
    import bench
    import workloads
    costs = [bench.batch_cost(w["n1"]) for w in workloads.const_1d_batch()]
    assert bench.shard_by_cost(costs, 1) == [list(range(len(costs)))]
    for world in (2, 3, 4, 8):
        parts = bench.shard_by_cost(costs, world)
        assert sorted(i for p in parts for i in p) == list(range(len(costs)))
        assert all(p == sorted(p) for p in parts)
        loads = [sum(costs[i] for i in p) for p in parts]
        # longest-first greedy: no rank exceeds the mean by more than one instance's cost
        assert max(loads) <= sum(costs) / world + max(costs)
        assert max(loads) / (sum(costs) / world) < 1.01


def test_cpu_baseline_times_the_oracle_at_one_and_all_threads():
    """The CPU baseline: the oracle's own solve of the n = 1023 PCG system,
    at one FFT thread and at two, reported as solves/s with the threads used."""
    sys.path.insert(0, ROOT)
    import bench
    s = bench.cpu_sample("latency1d", 1, 500)
    assert s["solves"] == 1 and 1 <= s["iterations"] < 20 and s["seconds"] > 0
    r = bench.cpu_baseline("latency1d", float(s["iterations"]), 500, 2)
    assert r["kind"] == "oracle" and r["cores"] == 1 and r["value"] > 0
    assert r["all_cores"]["cores"] == 2 and r["all_cores"]["value"] > 0


def test_algorithmic_flop_counts_match_the_hand_counts():
    """The bench's FFT flop accounting against counts made by hand from the
    transforms per iteration: n = 65535 GMRES about 28 MFLOP; 2047^2 PCG
    about 2.0 GFLOP; 4095^2 GMRES about 10.9 GFLOP."""
    sys.path.insert(0, ROOT)
    import bench
    g1 = bench.Geometry(1, 65535, 1, "gmres", True, 2)
    assert g1.transform_flops() == pytest.approx(27.85e6, rel=1e-3)
    assert bench.Geometry(2, 2047, 2047, "pcg", False, 0).transform_flops() == pytest.approx(2.013e9, rel=1e-3)
    assert bench.Geometry(2, 4095, 4095, "gmres", True, 4).transform_flops() == pytest.approx(10.90e9, rel=1e-3)
    r = bench.alu_roofline(10.90e9, 1000.0, bench.FP64_PEAK_TFLOPS)
    assert r["bound"] == "alu" and r["achieved"] == pytest.approx(10.90e9 / 1e12)
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(1.25856)


def test_algorithmic_byte_count_matches_an_enumeration_of_the_passes():
    """One full GMRES(20) cycle on the 4095^2 plane (20 steps, D_N and four
    coefficient arrays), counted vector pass by vector pass: forming V_j reads
    w and j basis vectors and writes V_j; the tau solve reads V_j and D^-1 and
    writes z; the matvec reads z and four coefficient arrays and writes w; the
    dots read w and j + 1 basis vectors; the cycle's residual reads x, b and
    the coefficient arrays and writes V_0, its norm reads V_0, the update reads
    20 basis vectors, D^-1 and x and writes x."""
    sys.path.insert(0, ROOT)
    import bench
    m = 20
    passes = 0
    for j in range(m):
        if j >= 1:
            passes += 1 + j + 1
        passes += 3 + 6 + (j + 2)
    passes += (1 + 1 + 4 + 1) + 1 + (m + 1 + 2)
    N = 4095 * 4095
    g = bench.Geometry(2, 4095, 4095, "gmres", True, 4)
    info = dict(iterations=m, cycles=1, basis_sum=sum(j + 1 for j in range(m)), residuals64=0, iterations64=m)
    assert bench.solve_bytes(info, g, 8) == pytest.approx(passes * 8 * N)
    info32 = dict(info, iterations64=0)
    assert bench.solve_bytes(info32, g, 4) == pytest.approx(passes * 4 * N)


def test_kappa_estimate_orders_the_alphas_and_the_rule_splits_them():
    """The symbol-based kappa(M) estimate grows with alpha on the 1D march
    (about h^-alpha), and the u32 kappa rule keeps FP32 inner solves for
    alpha = 1.2 only; against a dense condition number at small n the
    estimate is an upper bound within two orders."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    import oracle
    import workloads
    ws = workloads.var_1d_time_stepping(n=65535, alphas=(1.2, 1.5, 1.8), steps=2)
    ks = [bench.kappa_estimate(w) for w in ws]
    assert ks[0] < ks[1] < ks[2]
    fake = {"f64": {"per_alpha": {str(w["alpha"]): {"iterations": 1} for w in ws}}}
    choice = {a: v["choice"] for a, v in bench.precision_by_alpha(ws, fake).items()}
    assert choice == {"1.2": "f32_ir", "1.5": "f64", "1.8": "f64"}
    w = workloads.var_1d_time_stepping(n=255, alphas=(1.5,), steps=2)[0]
    n = w["n1"]
    h = w["length"] / (n + 1)
    prob = oracle.Problem1D(alpha=1.5, n=n, c0=h ** 1.5 / w["dt"], dp=w["dp"], dm=w["dm"])
    kd = np.linalg.cond(prob.dense())
    ke = bench.kappa_estimate(w)
    assert kd <= ke * 1.01 and ke <= 100 * kd, (kd, ke)


def test_measured_traffic_scales_by_units_and_drops_a_stale_capture(tmp_path, monkeypatch):
    """roofline.traffic: DRAM bytes per unit of algorithmic bytes from the
    capture, times the reporting launch's units; None once the sources'
    hash differs from the capture's, or without a capture."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    (tmp_path / "profiles").mkdir()
    h = bench.source_hash()
    tab = {"k:now": {"source_hash": h, "dram_bytes": 30.0, "units": 10.0},
           "k:old": {"source_hash": "0" * 16, "dram_bytes": 30.0, "units": 10.0}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(tab))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_hash", lambda: h)
    assert bench.measured_traffic("k:now", 7.0) == 21.0
    assert bench.measured_traffic("k:old", 7.0) is None
    assert bench.measured_traffic("k:none", 7.0) is None


def test_both_arms_name_the_same_headline_config():
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    a = argparse.Namespace(steps=47, warmup=3)
    c = bench.headline_config(a)
    assert c == bench.headline_config(argparse.Namespace(steps=47, warmup=3))
    assert c["workload"] == "2d-var-n4095-50steps-gmres20" and c["unknowns"] == 4095 * 4095
    assert c["march"].startswith("steps 4..50 ")
