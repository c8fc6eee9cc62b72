"""The multi-rank bench logic on CPU: world size 2 over gloo.

bench.py under torchrun gives every rank an independent copy of the
workload (its own seeded test block), times it, and reduces the elapsed time
with a MAX over ranks; the job throughput is ranks x per-rank actions over
that maximum.  These tests run the same helpers in two gloo processes.
"""
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


def _worker(rank, world, port, results):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    elapsed = 1.0 + rank          # rank 1 is the slow one
    t = bench.max_over_ranks(elapsed)
    results[rank] = (t, bench.job_throughput(100.0, ws, t), bench.rank_seed_offset(rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_time_and_weak_scaling():
    world, port = 2, _free_port()
    mgr = mp.Manager()
    results = mgr.dict()
    mp.spawn(_worker, args=(world, port, results), nprocs=world, join=True)
    assert results[0][0] == results[1][0] == 2.0       # max over ranks
    assert results[0][1] == results[1][1] == 100.0     # 2 ranks x 100 actions / 2 s
    assert results[0][2] != results[1][2]              # independent test blocks per rank


def test_rank_blocks_are_independent():
    import numpy as np
    import bench
    import workloads as W
    w = W.small_gl()
    a = W.test_block(w, seed_offset=bench.rank_seed_offset(0))
    b = W.test_block(w, seed_offset=bench.rank_seed_offset(1))
    assert a.shape == b.shape and not np.allclose(a, b)

