"""The multi-process host logic of bench.py on CPU (gloo, world size 2).

The hot path does not shard (one geometry per GPU), so several GPUs run
independent replicas; what the ranks share is the timing: a barrier around
the timed region and the maximum of the per-rank times (the job's time), from
which the whole-job rate is computed. This runs that logic with two gloo
ranks on the host."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        bench._barrier(world)
        t = bench._max_over_ranks(10.0 * (rank + 1), world, torch.device("cpu"))
        bench._barrier(world)
        results[rank] = t
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_barrier_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    results = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, results)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    # every rank sees the slowest rank's time
    assert dict(results) == {0: 20.0, 1: 20.0}


def test_single_rank_needs_no_process_group():
    import bench
    assert bench._max_over_ranks(3.5, 1, None) == 3.5
    bench._barrier(1)
    ws, rank, local = bench._dist()
    assert ws >= 1 and 0 <= rank < ws and local >= 0
