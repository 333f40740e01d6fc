"""The N > 1 bench path on CPU: two gloo ranks aggregate their replica
timings as the GPU ranks do (units of all ranks over the slowest rank's
time), and a rank that never joins ends the rendezvous with an error."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, units, ms, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        value, tmax = bench.aggregate(units[rank], ms[rank], dist, torch.device("cpu"))
        out[rank] = (value, tmax)
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregate():
    units, ms = [1000.0, 3000.0], [20.0, 50.0]
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(2, _free_port(), units, ms, out), nprocs=2, start_method="spawn")
        res = dict(out)
    for rank in (0, 1):
        value, tmax = res[rank]
        assert tmax == 50.0
        assert abs(value - 4000.0 / 0.05) < 1e-6


def test_single_rank_aggregate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(500.0, 10.0, None, None) == (50000.0, 10.0)


def _lonely(rank, port, out):
    from datetime import timedelta
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    try:
        dist.init_process_group("gloo", rank=rank, world_size=2, timeout=timedelta(seconds=3))
        dist.barrier()
        out[rank] = "joined"
    except Exception as e:  # the peer never arrives
        out[rank] = type(e).__name__


def test_missing_rank_fails_the_rendezvous():
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_lonely, args=(_free_port(), out), nprocs=1, start_method="spawn")
        assert out[0] != "joined"
