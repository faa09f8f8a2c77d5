"""The N > 1 path of bench.py on CPU: two gloo ranks, replicas only.

Each rank reports its own work and times; the bench line must carry the sum
of the work and the maximum of the times over ranks (weak scaling, no data
path collective).
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    work = [1.0e9, 3.0e9][rank]
    pcg = [10.0, 25.0][rank]
    tot = [100.0, 80.0][rank]
    out[rank] = bench.reduce_ranks(dist, work, pcg, tot, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    for r in range(2):
        assert out[r] == (4.0e9, 25.0, 100.0)
