"""bench.py's multi-rank logic on CPU: gloo, world_size 2 (no GPU).

Each rank answers its own query batch (weak scaling, no collective on the
data path); only timings are reduced, by a max over ranks.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, lr, w = bench.dist_env()
        assert (r, lr, w) == (rank, rank, world)
        got = bench.reduce_max([float(rank), 10.0 - rank, 3.5], world)
        bench.barrier(world)
        out[rank] = got
    finally:
        dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    for rank in range(world):
        assert out[rank] == [1.0, 10.0, 3.5]


def test_ranks_answer_distinct_query_batches():
    q0 = bench.queries_for_rank("c1", 0)
    q1 = bench.queries_for_rank("c1", 1)
    import workloads
    _, Q, _ = workloads.workload("c1")
    assert np.array_equal(q0, Q)  # rank 0 = the configuration's queries
    assert q1.shape == q0.shape and not np.array_equal(q0, q1)


def test_single_rank_reduce_is_identity():
    assert bench.reduce_max([1.0, 2.0], 1) == [1.0, 2.0]
