"""The benchmark's multi-process path on the CPU (gloo, world size 2).

Multi-GPU runs are replicas: each rank solves its own propagators, the only
cross-rank steps are barriers around the timed region and the maximum of the
per-rank times.  These run here with the gloo backend and no GPU.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), LQCD_DIST_BACKEND="gloo")
    import bench
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    t = bench.max_over_ranks(1.5 + rank, w)  # rank 1 is the slower one
    out[rank] = t
    bench.barrier(w)
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_replica_timing_takes_the_max_over_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    assert out[0] == out[1] == 2.5
