"""Multi-rank host logic of bench.py, on CPU with gloo (world size 2).

The apply does not shard: under torchrun every rank runs an independent
replica on its own point set, the job's time is the slowest rank's, and the
reported value sums the replicas' work. These tests run that aggregation on
two gloo ranks, and check that the reference arm's non-zero ranks exit
without work.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = [12.5, 20.0][rank]
        dist.barrier()
        ms = bench.max_over_ranks(ms_local, dist, torch.device("cpu"))
        value = bench.whole_job_value(1 << 20, 32, world, ms)
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.replica_seed(1, rank))
        ret = None
        if rank == 1:
            # the reference arm does its work on rank 0 only
            ret = bench.run_reference(type("A", (), {"n": None, "warmup": 0, "steps": 0, "gpus": world})())
        out.put((rank, ms, value, seeds, ret))
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        r = q.get(timeout=120)
        res[r[0]] = r
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        _, ms, value, seeds, _ = res[r]
        assert ms == 20.0                                 # slowest rank
        assert value == pytest.approx((1 << 20) * 32 * 2 / 20e-3 / 1e6)
        assert len(set(seeds)) == 2                       # independent replicas
    assert res[1][4] == 0                                 # reference arm: rank 1 returns at once
