"""The multi-GPU bench path (independent replicas) on CPU: two gloo ranks.

bench.py under torchrun runs one replica per GPU and reports all ranks'
updates divided by the slowest rank's time.  The aggregation is checked here
with a world_size-2 gloo process group on 127.0.0.1.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.rank_max(1.0 + rank, dist, "cpu")            # rank 1 is the slower one
        rate = bench.whole_job_rate(1000.0, world, t)
        out.put((rank, t, rate))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_replica_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, rate in res:
        assert t == 2.0                                 # max over ranks
        assert rate == pytest.approx(1000.0 * 2 / 2.0)  # all ranks' units / slowest time


def test_single_process_needs_no_group():
    import bench
    assert bench.rank_max(3.5, None, "cpu") == 3.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
