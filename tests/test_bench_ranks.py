"""The bench's multi-process path on CPU: two gloo ranks (the GPU machine runs one NCCL rank per
GPU).  The runs are independent replicas with no collective on the data path; the only
collectives are the timing barrier and the max-over-ranks reduction of the timed region, and
the reported value is the units all ranks processed over the slowest rank's time."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, queue):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(10.0 + rank, dist, "cpu")   # rank 1 is the slow one
    dist.barrier()
    queue.put((rank, t))
    dist.destroy_process_group()


def test_whole_job_time_is_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    results = dict(queue.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert results == {0: 11.0, 1: 11.0}


def test_whole_job_rate_and_single_process():
    import bench
    assert bench.whole_job_rate(1000, 2, 5, 0.5) == 20000.0
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import argparse
    import bench
    args = argparse.Namespace(workload="twostream-32c-2M", steps=1, warmup=0, gpus=2)
    bench.run_reference(args, 2, 1)
    assert capsys.readouterr().out == ""
