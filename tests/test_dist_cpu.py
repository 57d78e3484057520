"""The N-GPU bench path is N independent replicas: a barrier, then the job's
time is the maximum over ranks and its rate counts every rank's points.
Checked with world_size 2 over gloo on the CPU (no GPU)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert bench.dist_env() == (world, rank, rank)
    dist.barrier()
    slow = bench.max_over_ranks(1.0 + rank, "cpu")  # rank 1 is the slow one
    rate = bench.whole_job_rate(world, 1000, slow)
    out.put((rank, slow, rate))
    dist.destroy_process_group()


def test_two_rank_max_and_weak_scaling_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[1] for r in res] == [2.0, 2.0]          # both see the slowest rank's time
    assert [r[2] for r in res] == [1000.0, 1000.0]    # 2 ranks x 1000 points / 2 s


def test_single_process_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.whole_job_rate(1, 500, 2.0) == 250.0
