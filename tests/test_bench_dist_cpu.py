"""bench.py's N > 1 path on the host: two gloo ranks (one process each, as
torchrun starts them) agree on the barrier and on the maximum time over ranks,
and only rank 0 runs the reference arm."""
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


def _rank(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    ws, r, _ = bench.dist_setup()
    bench.barrier(ws)
    # each rank's time differs; every rank must see the slowest
    out[r] = bench.max_over_ranks(ws, 1.5 + r)
    bench.barrier(ws)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        assert dict(out) == {0: 2.5, 1: 2.5}


def test_reference_arm_runs_on_rank_0_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, gpus = 1, 0, 2

    bench.run_reference(A(), 2, 1)  # rank 1: no work, no output
    assert capsys.readouterr().out == ""
