"""Multi-rank logic of bench.py on CPU (gloo, world size 2): the path
shards into independent replicas, so the only collective is the
max-over-ranks reduction of the timings, and the job value is all ranks'
steps over the slowest rank's time."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.init_dist()
    local_seconds = 1.0 + rank          # rank 1 is the slow one
    mx = bench.max_over_ranks(local_seconds)
    val = bench.replica_throughput(5, ws, mx)
    out[rank] = (ws, r, local, mx, val)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_is_max_over_ranks():
    import torch.multiprocessing as mp
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        ws, r, local, mx, val = out[rank]
        assert (ws, r, local) == (world, rank, rank)
        assert mx == 2.0
        assert val == pytest.approx(world * 5 / 2.0)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_throughput(4, 1, 2.0) == 2.0
