"""The multi-GPU path is replicas only: every rank tracks its own Time Frames
and the only collective is the max over ranks of the timed duration.  That
host logic runs here as two gloo ranks on the CPU (no GPU)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
        got = bench.device_max(ms, world, rank, device="cpu")
        seed = bench.replica_seed(20210609, rank)
        seeds = [None] * world
        dist.all_gather_object(seeds, seed)
        out[rank] = (got, seeds, bench.aggregate_rate(1000.0, world, got))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        got, seeds, rate = res[r]
        assert got == 150.0                      # max over ranks, on every rank
        assert len(set(seeds)) == world          # each replica its own TFs
        assert rate == pytest.approx(world * 1000.0 / 0.150)
