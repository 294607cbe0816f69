"""Autotuner of the enumerator's launch: block size, candidate-stack depth and
root-split threshold, picked per (k, degree profile) by timing candidates on
the device and cached as JSON.

The degree profile of a graph is the tuple (k, log2 n, log2 max degree, mean
undirected degree rounded, share of arcs at vertices of degree >= 32), so graphs
of one family (a null-model ensemble, a stream of similar requests) share one
entry.  Every candidate is checked against the automatic launch's histogram
before it can win, so tuning never changes results.
"""
from __future__ import annotations

import dataclasses
import json
import math
import os

import numpy as np

from . import count_stats, count_tuned, make_tuning, to_numpy_u64  # noqa: F401

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "motifs_gb300", "autotune.json")


@dataclasses.dataclass
class TuneParams:
    warps_per_block: int = 0
    split_scale: float = 0.0
    stack_cap: int = 0
    ms: float = float("nan")

    def tuning(self):
        return make_tuning(0.0, self.warps_per_block, self.split_scale, self.stack_cap)


def degree_profile(g, k: int) -> str:
    """Profile key of a synthetic.Graph-like object (n, row_ptr, col)."""
    src = np.repeat(np.arange(g.n), np.diff(np.asarray(g.row_ptr)))
    dst = np.asarray(g.col)
    lo, hi = np.minimum(src, dst), np.maximum(src, dst)
    pairs = np.unique(lo.astype(np.int64) * g.n + hi)
    deg = np.bincount(pairs // g.n, minlength=g.n) + np.bincount(pairs % g.n, minlength=g.n)
    dmax = int(deg.max()) if g.n else 0
    mean = float(deg.mean()) if g.n else 0.0
    hub = float(deg[deg >= 32].sum() / max(deg.sum(), 1))
    return (f"k{k}-n{int(round(math.log2(max(g.n, 1))))}-d{int(round(math.log2(max(dmax, 1))))}"
            f"-m{int(round(mean))}-h{int(round(10 * hub))}")


def candidates(max_degree: int, k: int):
    full = (k - 1) * max(max_degree, 1) + 32
    for wpb in (8, 16, 32):
        for scale in (0.25, 0.5, 1.0, 2.0, 8.0):
            for cap in (0, max(32, full // 2)):
                yield TuneParams(wpb, scale, cap)


def _time(fn, reps: int) -> float:
    import torch
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def tune(dev_graph, table, graph=None, reps: int = 3, cache_path: str | None = DEFAULT_CACHE,
         force: bool = False) -> TuneParams:
    """Best TuneParams for this graph's (k, degree profile); cached."""
    key = degree_profile(graph, table.k) if graph is not None else (
        f"k{table.k}-n{dev_graph.n}-d{dev_graph.max_degree}")
    cache = load_cache(cache_path)
    if not force and key in cache:
        return TuneParams(**cache[key])
    import torch
    ref = to_numpy_u64(count_tuned(dev_graph, table)).copy()
    base = TuneParams(0, 0.0, 0, _time(lambda: count_tuned(dev_graph, table), reps))
    best = base
    out = torch.empty(table.num_classes, dtype=torch.int64, device="cuda")
    for c in candidates(dev_graph.max_degree, table.k):
        def run(c=c):
            count_tuned(dev_graph, table, 0.0, c.warps_per_block, out, split_scale=c.split_scale,
                        stack_cap=c.stack_cap)
        run()
        torch.cuda.synchronize()
        if count_stats(dev_graph)[1] != 0:  # stack too shallow for this graph
            continue
        if not np.array_equal(to_numpy_u64(out), ref):
            raise RuntimeError(f"tuned launch {c} changed the histogram")
        c.ms = _time(run, reps)
        if c.ms < best.ms:
            best = c
    cache[key] = dataclasses.asdict(best)
    save_cache(cache, cache_path)
    return best


def tune_batch(dev_graph, table, graph, swaps: int, probe_nulls: int = 16, method: int = 0,
               reps: int = 2, cache_path: str | None = DEFAULT_CACHE,
               force: bool = False) -> TuneParams:
    """Best TuneParams for the null-model batch of this graph's degree profile,
    timed on a probe batch of `probe_nulls` null graphs (the counting phase,
    device events); every candidate's histograms must equal the automatic
    launch's."""
    import torch

    from . import Batch

    key = degree_profile(graph, table.k) + f"-batch-m{method}"
    cache = load_cache(cache_path)
    if not force and key in cache:
        return TuneParams(**cache[key])
    seeds = np.arange(1, probe_nulls + 1, dtype=np.uint64)
    ref = None
    best = None
    for wpb in (16, 32):
        for scale in (0.25, 0.5, 1.0, 2.0):
            c = TuneParams(wpb, scale, 0)
            tun = make_tuning(0.0, wpb, scale, 0, method)
            b = Batch(dev_graph, table, probe_nulls, swaps, tun)
            h, _ = b.run(seeds)
            torch.cuda.synchronize()
            if b.error() != 0:
                b.free()
                continue
            hn = to_numpy_u64(h).copy()
            if ref is None:
                ref = hn
            elif not np.array_equal(hn, ref):
                raise RuntimeError(f"tuned batch {c} changed the histograms")
            ts = []
            for _ in range(reps):
                b.run(seeds, h)
                ts.append(b.phase_ms()[1])
            c.ms = float(np.median(ts))
            b.free()
            if best is None or c.ms < best.ms:
                best = c
    cache[key] = dataclasses.asdict(best)
    save_cache(cache, cache_path)
    return best


def load_cache(path: str | None) -> dict:
    if not path or not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def save_cache(cache: dict, path: str | None) -> None:
    if not path:
        return
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
