"""Multi-process sharding on CPU (gloo, world size 2): each rank owns a
contiguous block of stream ids; the blocks generated independently, side by
side, are exactly the single-generator output (columns of one larger run),
so the path needs no data exchange.  The timing reduction the benchmark uses
(max over ranks) is exercised on the same process group."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import paper_1609_01257_gb300 as rng


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, total, seed, iters, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first, count = rng.shard_range(total, rank, world)
        block = oracle.generate(count, seed, iters, g0=first)
        parts = [None] * world
        dist.all_gather_object(parts, (first, block))
        t = torch.tensor([float(rank + 1)], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        if rank == 0:
            q.put((parts, float(t.item())))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("total", [1000, 4097])
def test_two_rank_shards_form_the_whole_generator(total):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    seed, iters = 12345, 6
    procs = [ctx.Process(target=_worker, args=(r, 2, port, total, seed, iters, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    parts.sort(key=lambda x: x[0])
    joined = np.concatenate([b for _, b in parts], axis=1)
    assert np.array_equal(joined, oracle.generate(total, seed, iters))
    assert tmax == 2.0
