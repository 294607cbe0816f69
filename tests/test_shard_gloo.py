"""The N>1 path on CPU: world-size-2 gloo ranks shard the null-model seeds and the
roots of one graph; the reduced histograms equal the one-rank result (oracle
counts stand in for the per-rank GPU counts, so this runs without a GPU)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import synthetic as syn
from paper_1804_09741_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # seeds: disjoint, together 1..R*world
        seeds = shard.rank_seeds(4, rank)
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds.tolist())
        # roots of one graph: ranges by estimated work, histograms add up
        g = syn.chung_lu_digraph(150, 500, 2.2, None, 0.1, 9)
        deg = np.zeros(g.n)
        s, d = g.arcs()
        for a, b in {(min(x, y), max(x, y)) for x, y in zip(s.tolist(), d.tolist())}:
            deg[a] += 1
            deg[b] += 1
        ranges = shard.root_ranges(deg ** 3, world)
        a, b = ranges[rank]
        h, _ = oracle.count_roots(g, 4, np.arange(a, b), nthreads=2)
        classes = sorted(oracle.count(g, 4, nthreads=2)[0])
        dense = np.array([h.get(c, 0) for c in classes], dtype=np.uint64)
        total = shard.reduce_histograms(dense, dist)
        t = shard.max_over_ranks(float(rank + 1), dist)
        if rank == 0:
            out.put((gathered, ranges, total.tolist(), t, classes))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import oracle
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, ranges, total, tmax, classes = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat = sorted(x for part in gathered for x in part)
    assert flat == list(range(1, 9))
    assert ranges[0][0] == 0 and ranges[-1][1] == 150 and ranges[0][1] == ranges[1][0]
    g = syn.chung_lu_digraph(150, 500, 2.2, None, 0.1, 9)
    want, _ = oracle.count(g, 4)
    assert total == [want[c] for c in classes]
    assert tmax == 2.0


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_root_ranges_cover_every_root_once(world):
    rng = np.random.default_rng(world)
    w = rng.pareto(1.5, size=97)
    r = shard.root_ranges(w, world)
    assert r[0][0] == 0 and r[-1][1] == 97
    assert all(r[i][1] == r[i + 1][0] for i in range(world - 1))
    assert shard.root_ranges(np.zeros(10), 3) == [(0, 3), (3, 6), (6, 10)]
