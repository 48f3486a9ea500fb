"""The multi-rank host logic of bench.py (replicas: one registration per rank, barrier and
max-over-ranks timing, no collective on the data path), run as two gloo ranks on CPU."""
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


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    # per-rank step times: the job's time is the slowest rank's
    t = bench.max_over_ranks(1.0 + rank * 0.5, world)
    bench.barrier(world)
    out[rank] = t
    dist.destroy_process_group()


def test_two_rank_timing_takes_the_slowest_rank():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res == {0: 1.5, 1: 1.5}


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5
    bench.barrier(1)
