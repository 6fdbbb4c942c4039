"""The N > 1 host path of bench.py on CPU: two gloo ranks, each with its own
replica's time and points; the job's time is the slowest rank's, its points
the sum (independent replicas, no data-path collective)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    t, p = bench.aggregate_replicas(10.0 * (rank + 1), 100.0 * (rank + 1), world, "cpu")
    out[rank] = (t, p)
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_replicas_gloo():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (20.0, 300.0)


def test_one_replica_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_replicas(3.5, 7.0, 1, "cpu") == (3.5, 7.0)
