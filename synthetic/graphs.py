"""Seeded generators of directed graphs in sorted int32 CSR form.

Every generator returns a :class:`Graph` whose ``row_ptr`` (n+1) and ``col`` (m)
describe the out-neighbours of each vertex, each row sorted ascending, with no
self-loops and no duplicate arcs.  Randomness comes only from
``numpy.random.Generator(PCG64(seed))``.

Readings of the paper's unstated workload details (the paper's datasets,
Table 2, are not available, so these stand in for them):

* uniform graph: G(n, M), M distinct ordered pairs u != v drawn uniformly;
* Chung-Lu graph: expected-degree weights w_i proportional to (i+1)^(-1/(gamma-1)),
  scaled so that sum(w) = m and clipped at ``dmax`` (then rescaled, clipping
  again, until the sum settles); in-weights are an independent seeded
  permutation of the same sequence; round(r*m/2) mutual pairs are drawn first,
  then single arcs, with tails drawn by out-weight and heads by in-weight;
  self-loops and pairs already present in either direction are rejected.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Graph:
    """A directed graph as a sorted CSR of out-neighbours."""

    n: int
    row_ptr: np.ndarray  # int32[n+1]
    col: np.ndarray  # int32[m]
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.col.shape[0])

    def arcs(self) -> tuple[np.ndarray, np.ndarray]:
        src = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.row_ptr))
        return src, self.col.astype(np.int64)


def csr_from_arcs(n: int, src, dst, name: str = "") -> Graph:
    """Sorted CSR from arc lists (duplicates are kept; callers pass distinct arcs)."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    counts = np.bincount(src, minlength=n) if n > 0 else np.zeros(0, np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(counts)
    return Graph(n, row_ptr.astype(np.int32), dst.astype(np.int32), name)


# --------------------------------------------------------------------------- workloads


def uniform_digraph(n: int, m: int, seed: int) -> Graph:
    """G(n, M): ``m`` distinct ordered pairs (u, v), u != v, uniform."""
    if m > n * (n - 1):
        raise ValueError("too many arcs")
    rng = np.random.Generator(np.random.PCG64(seed))
    seen: set[tuple[int, int]] = set()
    src, dst = [], []
    while len(src) < m:
        need = m - len(src)
        u = rng.integers(0, n, size=2 * need + 16)
        v = rng.integers(0, n, size=2 * need + 16)
        for a, b in zip(u.tolist(), v.tolist()):
            if a == b or (a, b) in seen:
                continue
            seen.add((a, b))
            src.append(a)
            dst.append(b)
            if len(src) == m:
                break
    return csr_from_arcs(n, src, dst, f"uniform(n={n},m={m},seed={seed})")


def _chung_lu_weights(n: int, m: int, gamma: float, dmax: float | None) -> np.ndarray:
    i = np.arange(n, dtype=np.float64)
    w = (i + 1.0) ** (-1.0 / (gamma - 1.0))
    w *= m / w.sum()
    if dmax is not None:
        for _ in range(200):
            w = np.minimum(w, float(dmax))
            s = w.sum()
            if abs(s - m) <= 1e-9 * m:
                break
            free = w < dmax
            if not free.any():
                break
            w[free] *= (m - w[~free].sum()) / w[free].sum()
    return w


def chung_lu_digraph(n: int, m: int, gamma: float, dmax: float | None, recip: float,
                     seed: int) -> Graph:
    """Directed Chung-Lu graph with exactly ``m`` arcs and reciprocity ~``recip``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w_out = _chung_lu_weights(n, m, gamma, dmax)
    w_in = w_out[rng.permutation(n)]
    p_out = w_out / w_out.sum()
    p_in = w_in / w_in.sum()
    und: set[tuple[int, int]] = set()
    src: list[int] = []
    dst: list[int] = []
    n_mutual = int(round(recip * m / 2.0))

    def draw(count: int):
        a = rng.choice(n, size=count, p=p_out)
        b = rng.choice(n, size=count, p=p_in)
        return a.tolist(), b.tolist()

    guard = 0
    while len(src) < 2 * n_mutual:
        guard += 1
        if guard > 10000:
            raise RuntimeError("could not place mutual pairs")
        for a, b in zip(*draw(2 * (2 * n_mutual - len(src)) + 16)):
            if a == b:
                continue
            key = (a, b) if a < b else (b, a)
            if key in und:
                continue
            und.add(key)
            src += [a, b]
            dst += [b, a]
            if len(src) >= 2 * n_mutual:
                break
    while len(src) < m:
        guard += 1
        if guard > 20000:
            raise RuntimeError("could not place single arcs")
        for a, b in zip(*draw(2 * (m - len(src)) + 16)):
            if a == b:
                continue
            key = (a, b) if a < b else (b, a)
            if key in und:
                continue
            und.add(key)
            src.append(a)
            dst.append(b)
            if len(src) >= m:
                break
    g = csr_from_arcs(n, src, dst)
    g.name = f"chung_lu(n={n},m={m},gamma={gamma},dmax={dmax},r={recip},seed={seed})"
    return g


# The paper's workloads as synthetic stand-ins (sizes of Table 2's networks).
WORKLOADS = {
    "uniform_k3": dict(kind="uniform", n=300, m=1500, seed=0, k=3),
    "chunglu_k4": dict(kind="chung_lu", n=2000, m=8000, gamma=2.3, dmax=150, recip=0.15,
                       seed=0, k=4),
    "nullmodel_k5": dict(kind="chung_lu", n=1500, m=6000, gamma=2.2, dmax=None, recip=0.10,
                         seed=0, k=5, nulls=256),
    "nullmodel_k6": dict(kind="chung_lu", n=800, m=3200, gamma=2.5, dmax=40, recip=0.10,
                         seed=0, k=6, nulls=64),
}


def workload_graph(name: str) -> Graph:
    """The original graph of a named workload."""
    w = WORKLOADS[name]
    if w["kind"] == "uniform":
        return uniform_digraph(w["n"], w["m"], w["seed"])
    return chung_lu_digraph(w["n"], w["m"], w["gamma"], w["dmax"], w["recip"], w["seed"])


def serving_stream(num: int, seed: int, nmax: int = 20000):
    """A seeded stream of count requests (k, graph, arrival gap in units of 1/rate).

    k is drawn from {3,4,5,6} with weights .2/.3/.3/.2; n log-uniform in
    [100, nmax] (at most 1,000 for k=6); mean out-degree U[2,8]; gamma U[2.1,2.8];
    reciprocity U[0,0.3]; per-direction degree cap 150/150/60/40 for k=3/4/5/6.
    The caller redraws requests whose work bound is too large.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    caps = {3: 150, 4: 150, 5: 60, 6: 40}
    out = []
    for i in range(num):
        k = int(rng.choice([3, 4, 5, 6], p=[0.2, 0.3, 0.3, 0.2]))
        hi = min(nmax, 1000) if k == 6 else nmax
        n = int(round(math.exp(rng.uniform(math.log(100), math.log(hi)))))
        deg = float(rng.uniform(2.0, 8.0))
        gamma = float(rng.uniform(2.1, 2.8))
        recip = float(rng.uniform(0.0, 0.3))
        m = int(round(deg * n))
        gap = float(rng.exponential(1.0))
        g = chung_lu_digraph(n, m, gamma, caps[k], recip, seed * 100003 + i)
        out.append((k, g, gap))
    return out


# --------------------------------------------------------------------------- fixtures


def random_small_digraph(n: int, p: float, recip: float, seed: int) -> Graph:
    """Dense-ish small digraph for brute-force checks: each ordered pair is an arc
    with probability p; a present arc's reverse is added with probability recip."""
    rng = np.random.Generator(np.random.PCG64(seed))
    adj = rng.random((n, n)) < p
    np.fill_diagonal(adj, False)
    rev = (rng.random((n, n)) < recip) & adj
    adj |= rev.T
    np.fill_diagonal(adj, False)
    s, d = np.nonzero(adj)
    return csr_from_arcs(n, s, d, f"small(n={n},p={p},seed={seed})")


def complete_digraph(n: int) -> Graph:
    s, d = np.nonzero(~np.eye(n, dtype=bool))
    return csr_from_arcs(n, s, d, f"complete({n})")


def empty_graph(n: int) -> Graph:
    return csr_from_arcs(n, [], [], f"empty({n})")


def directed_cycle(n: int) -> Graph:
    s = np.arange(n)
    return csr_from_arcs(n, s, (s + 1) % n, f"cycle({n})")


def bidirected_path(n: int) -> Graph:
    s = np.arange(n - 1)
    return csr_from_arcs(n, np.concatenate([s, s + 1]), np.concatenate([s + 1, s]),
                         f"bipath({n})")


def out_star(n: int) -> Graph:
    return csr_from_arcs(n, np.zeros(n - 1, np.int64), np.arange(1, n), f"outstar({n})")


def disjoint_union(g1: Graph, g2: Graph) -> Graph:
    s1, d1 = g1.arcs()
    s2, d2 = g2.arcs()
    return csr_from_arcs(g1.n + g2.n, np.concatenate([s1, s2 + g1.n]),
                         np.concatenate([d1, d2 + g1.n]), f"{g1.name}+{g2.name}")


def relabel(g: Graph, perm) -> Graph:
    """Vertex v becomes perm[v]."""
    perm = np.asarray(perm, dtype=np.int64)
    s, d = g.arcs()
    return csr_from_arcs(g.n, perm[s], perm[d], f"relabel({g.name})")


def reverse(g: Graph) -> Graph:
    s, d = g.arcs()
    return csr_from_arcs(g.n, d, s, f"reverse({g.name})")
