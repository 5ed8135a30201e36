"""The multi-rank host logic of bench.py (replicas, no collective on the data
path): with world_size 2 over gloo on the CPU, the job time is the maximum over
ranks, the work is the sum, and the barrier lets every rank through."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, l = bench.dist_env()
        assert (w, r, l) == (ws, rank, rank)
        bench.barrier(ws)
        t = bench.reduce_max(1.5 + rank, ws)          # rank 1 is the slow one
        n = bench.reduce_sum(100.0 * (rank + 1), ws)
        bench.barrier(ws)
        out[rank] = (t, n)
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_take_max_time_and_sum_work():
    ws = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
    assert out[0] == out[1] == (2.5, 300.0)


def test_single_rank_is_the_identity():
    import bench
    assert bench.reduce_max(3.0, 1) == 3.0 and bench.reduce_sum(7.0, 1) == 7.0
    bench.barrier(1)
