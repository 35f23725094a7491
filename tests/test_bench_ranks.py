"""Host logic of the multi-GPU bench on CPU, world size 2 over gloo.

The path shards into independent replicas (one per GPU, no data-path
collective): the job's time is the slowest rank's, its throughput the ranks'
combined work over that time.  These run without a GPU.
"""

import os
import socket

import pytest

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, queue):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench._max_over_ranks(1.0 + rank, dist, "cpu")     # rank r took 1 + r ms per step
        v = bench._job_value(world, 2.0e9, t)
        dist.barrier()
        queue.put((rank, t, v))
    finally:
        dist.destroy_process_group()


def test_two_replicas_time_is_the_slowest_rank_and_value_the_whole_job():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(queue.get(timeout=10) for _ in range(2))
    for rank, t, v in got:
        assert t == 2.0                                           # max over ranks on every rank
        assert v == pytest.approx(2 * 2.0e9 / 2.0e-3 / 1e9)       # two replicas' work in the slowest time


def test_single_process_is_the_identity():
    import torch.distributed as dist
    assert bench._max_over_ranks(3.5, dist, "cpu") == 3.5
    assert bench._job_value(1, 1.0e9, 1.0) == pytest.approx(1000.0)
