"""The N>1 path of bench.py (independent replicas, one per GPU) on CPU: two
gloo ranks check the cross-rank reductions the benchmark uses (slowest rank's
time, sum of edges) and the reference arm's rank-0-only rule."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import bench
    r, w, local = bench.dist_setup()
    assert (r, w) == (rank, ws)
    t = bench.max_over_ranks(1.0 + rank, w)          # per-rank time
    e = bench.sum_over_ranks(100.0 * (rank + 1), w)  # per-rank edges
    bench.barrier(w)
    out[rank] = (t, e)
    dist.destroy_process_group()


def test_two_gloo_replicas_reduce_like_the_benchmark():
    ws = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()  # no fork of a process that may hold a CUDA context
    out = mgr.dict()
    mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
    for rank in range(ws):
        t, e = out[rank]
        assert t == 2.0      # the slowest rank's time
        assert e == 300.0    # edges of all ranks


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.dist_setup() == (0, 1, 0) or int(os.environ.get("WORLD_SIZE", "1")) > 1
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.sum_over_ranks(7.0, 1) == 7.0
