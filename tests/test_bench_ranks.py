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
