"""The N > 1 layout on CPU with two gloo ranks: each rank transforms its own
batch (distinct seeds, rows covered exactly once when a global batch is
split) and the step time reported is the maximum over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1907_07875_gb300 import sharding


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = sharding.max_over_ranks(10.0 + rank, dist)
        seeds = [None] * world
        dist.all_gather_object(seeds, sharding.rank_seed(1002, rank))
        rows = [None] * world
        dist.all_gather_object(rows, sharding.shard_rows(1001, rank, world))
        out.put((rank, t, seeds, rows))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, seeds, rows in res:
        assert t == 11.0                       # max over ranks
        assert len(set(seeds)) == 2            # distinct per-rank batches
        covered = [i for a, b in rows for i in range(a, b)]
        assert covered == list(range(1001))    # split covers every row once


def test_single_process_identity():
    assert sharding.max_over_ranks(3.5) == 3.5
    assert sharding.shard_rows(10, 0, 1) == (0, 10)
