"""The bench's multi-rank timing aggregation (max of per-rank times, sum of
per-rank work) on two gloo ranks on the CPU; the data path itself has no
collective (replicas)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_setup()
    t_max, e_max = bench.aggregate([10.0 + rank, 3.0 * (rank + 1)], "max")
    units = bench.aggregate([float(100 * (rank + 1))], "sum")[0]
    out[rank] = (ws, r, t_max, e_max, units)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    import torch.multiprocessing as mp
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    for rank in (0, 1):
        ws, r, t_max, e_max, units = out[rank]
        assert (ws, r) == (2, rank)
        assert t_max == 11.0 and e_max == 6.0 and units == 300.0


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate([1.5, 2.5], "max") == [1.5, 2.5]
    assert bench.dist_setup()[0] >= 1
