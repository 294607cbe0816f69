"""Host-side sharding of the Motifs-k work across ranks (one GPU per rank).

Two partitions of the work exist, and neither needs a collective on the data
path:
* the null-model batch: graphs are independent, so rank r randomises and counts
  its own null graphs (seeds disjoint across ranks);
* one large graph: connected k-sets are owned by their smallest vertex, so
  disjoint root ranges give histograms that add up to the whole one; only the
  final uint64 histogram is reduced.
"""
from __future__ import annotations

import numpy as np


def rank_seeds(nulls_per_rank: int, rank: int, first_seed: int = 1) -> np.ndarray:
    """Seeds of rank `rank`: first_seed + rank*R ... first_seed + (rank+1)*R - 1."""
    base = first_seed + rank * nulls_per_rank
    return np.arange(base, base + nulls_per_rank, dtype=np.uint64)


def root_ranges(work_per_root, world: int) -> list[tuple[int, int]]:
    """Cut roots 0..n-1 into `world` contiguous ranges of about equal total work
    (any non-negative per-root estimate, e.g. sum of C(d, k-1) over the root's
    forward neighbourhood); every root lands in exactly one range."""
    w = np.asarray(work_per_root, dtype=np.float64)
    n = w.size
    total = float(w.sum())
    cuts = [0]
    if total <= 0.0:
        for r in range(1, world):
            cuts.append(n * r // world)
    else:
        csum = np.cumsum(w)
        for r in range(1, world):
            cuts.append(int(np.searchsorted(csum, total * r / world, side="left")) + 1)
    cuts.append(n)
    cuts = [min(max(c, 0), n) for c in cuts]
    for i in range(1, len(cuts)):
        cuts[i] = max(cuts[i], cuts[i - 1])
    return [(cuts[i], cuts[i + 1]) for i in range(world)]


def reduce_histograms(hist: np.ndarray, dist) -> np.ndarray:
    """Sum uint64 histograms over ranks (int64 transport: counts stay below 2^63)."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(hist).view(np.int64).copy())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.numpy().view(np.uint64)


def max_over_ranks(value: float, dist) -> float:
    import torch
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
