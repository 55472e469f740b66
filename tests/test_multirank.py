"""Multi-rank host logic on CPU (gloo, world size 2): batch sharding and the
max-over-ranks step time that bench.py reports."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2606_24039_gb300.shard import instance_work, lpt_shards, shard_of


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_lpt_shards_cover_the_batch_once_and_balance():
    rng = np.random.default_rng(0)
    N = rng.integers(10, 201, size=4096)
    n = rng.choice([6, 8, 8, 8], size=4096)
    work = instance_work(N, n)
    for world in (1, 2, 3, 8):
        parts = lpt_shards(work, world)
        allidx = np.concatenate(parts)
        assert np.array_equal(np.sort(allidx), np.arange(4096))
        loads = np.array([work[p].sum() for p in parts])
        # LPT: the spread of the loads is at most the largest single item
        assert loads.max() - loads.min() <= work.max() + 1e-9


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    from paper_2606_24039_gb300.shard import max_over_ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(1)
        work = instance_work(rng.integers(10, 201, size=100), 8)
        mine = shard_of(work, world, rank)
        ms = 10.0 + 5.0 * rank                 # the slower rank sets the job time
        q.put((rank, mine.tolist(), max_over_ranks(ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_disjointly_and_agree_on_the_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out.sort()
    a, b = set(out[0][1]), set(out[1][1])
    assert not (a & b) and len(a | b) == 100
    assert out[0][2] == out[1][2] == 15.0
