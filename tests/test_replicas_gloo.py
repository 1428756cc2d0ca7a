"""Multi-GPU runs of bench.py are independent replica streams (the stream of
frames is sequential and does not shard): the only cross-rank steps are the
barrier and the max-over-ranks of the timed region.  These run as two gloo
ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        mx = bench.barrier_max(10.0 + 5.0 * rank, world)
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.replica_seed(rank))
        out[rank] = (mx, seeds)
    finally:
        dist.destroy_process_group()


def test_two_rank_barrier_max_and_independent_replicas():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    # every rank sees the slowest rank's time
    assert res[0][0] == res[1][0] == 15.0
    # each rank reconstructs its own stream
    seeds = res[0][1]
    assert len(set(seeds)) == world and res[1][1] == seeds


def test_reference_arm_only_rank0_prints(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class A:
        warmup, steps = 0, 1

    assert bench.run_reference(A()) is None
    assert capsys.readouterr().out == ""
