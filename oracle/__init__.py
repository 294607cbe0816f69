"""Oracle for the Motifs-k hot path: plain, slow, obviously correct CPU code.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  Nothing here is shared with
the CUDA path; the two meet only through the seeded inputs of ``synthetic``.

Contents
--------
* ``oracle.cc`` (built into ``_build/liboracle.so``): brute-force canonical
  forms, ESU and brute-force-subset histograms, the sequential arc-swap
  randomiser and SplitMix64 (see the file header for the citations).
* :func:`zscores` here: per-class z-scores of Sec. 1 step (c) in float64.

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
library routines and brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``oracle.cc`` into ``_build/liboracle.so`` (g++ -O2, pthreads)."""
    src = os.path.join(_HERE, "oracle.cc")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-pthread",
                           src, "-o", tmp])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.POINTER
            i32p, u32p, u64p = P(ctypes.c_int32), P(ctypes.c_uint32), P(ctypes.c_uint64)
            lib.oracle_splitmix64.restype = ctypes.c_uint64
            lib.oracle_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.oracle_bit_index.restype = ctypes.c_int
            lib.oracle_bit_index.argtypes = [ctypes.c_int] * 3
            lib.oracle_canon.restype = ctypes.c_uint32
            lib.oracle_canon.argtypes = [ctypes.c_int, ctypes.c_uint32]
            lib.oracle_canon_many.restype = None
            lib.oracle_canon_many.argtypes = [ctypes.c_int, u32p, u32p, ctypes.c_int64,
                                              ctypes.c_int]
            lib.oracle_connected.restype = ctypes.c_int
            lib.oracle_connected.argtypes = [ctypes.c_int, ctypes.c_uint32]
            lib.oracle_class_masks.restype = ctypes.c_int64
            lib.oracle_class_masks.argtypes = [ctypes.c_int, ctypes.c_int, u32p, ctypes.c_int64,
                                               ctypes.c_int]
            lib.oracle_count.restype = ctypes.c_int64
            lib.oracle_count.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int, ctypes.c_int,
                                         u32p, u64p, ctypes.c_int64, u64p]
            lib.oracle_count_roots.restype = ctypes.c_int64
            lib.oracle_count_roots.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int, i32p,
                                               ctypes.c_int64, ctypes.c_int, u32p, u64p,
                                               ctypes.c_int64, u64p]
            lib.oracle_count_roots_split.restype = ctypes.c_int64
            lib.oracle_count_roots_split.argtypes = lib.oracle_count_roots.argtypes
            lib.oracle_count_connected_sets.restype = ctypes.c_uint64
            lib.oracle_count_connected_sets.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int,
                                                        ctypes.c_int]
            lib.oracle_count_bruteforce.restype = ctypes.c_int64
            lib.oracle_count_bruteforce.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int,
                                                    u32p, u64p, ctypes.c_int64, u64p]
            lib.oracle_randomize_dyads.restype = ctypes.c_int64
            lib.oracle_randomize_dyads.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_uint64,
                                                   ctypes.c_uint64, i32p, i32p]
            lib.oracle_randomize.restype = ctypes.c_int64
            lib.oracle_randomize.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_uint64,
                                             ctypes.c_uint64, i32p, i32p]
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, np.int32)
    return rp, col


_CAP = 1_600_000  # more than the 1,540,944 classes of all 6-vertex digraphs


def splitmix64(seed: int, i: int) -> int:
    """Output ``i`` (0-based) of SplitMix64 seeded with ``seed``."""
    return int(_load().oracle_splitmix64(seed, i))


def bit_index(k: int, i: int, j: int) -> int:
    return int(_load().oracle_bit_index(k, i, j))


def canon(k: int, mask: int) -> int:
    """Smallest mask over all k! relabellings (brute force)."""
    return int(_load().oracle_canon(k, mask))


def canon_many(k: int, masks, nthreads: int | None = None) -> np.ndarray:
    masks = np.ascontiguousarray(masks, dtype=np.uint32)
    out = np.empty_like(masks)
    _load().oracle_canon_many(k, _p(masks, ctypes.c_uint32), _p(out, ctypes.c_uint32),
                              masks.size, nthreads or default_threads())
    return out


def connected(k: int, mask: int) -> bool:
    return bool(_load().oracle_connected(k, mask))


def class_masks(k: int, connected_only: bool = True, nthreads: int | None = None) -> np.ndarray:
    """All canonical masks (k <= 5), ascending; index = dense class id."""
    out = np.empty(_CAP, np.uint32)
    cnt = _load().oracle_class_masks(k, int(connected_only), _p(out, ctypes.c_uint32), _CAP,
                                     nthreads or default_threads())
    if cnt < 0:
        raise ValueError("k must be in 2..5")
    return out[:cnt].copy()


def _hist_call(fn, *args):
    masks = np.empty(_CAP, np.uint32)
    counts = np.empty(_CAP, np.uint64)
    sets = ctypes.c_uint64(0)
    cnt = fn(*args, _p(masks, ctypes.c_uint32), _p(counts, ctypes.c_uint64), _CAP,
             ctypes.byref(sets))
    if cnt < 0:
        raise ValueError("bad arguments")
    return dict(zip(masks[:cnt].tolist(), counts[:cnt].tolist())), int(sets.value)


def count(g, k: int, nthreads: int | None = None):
    """H_k(G) as {canonical mask: count} and the number of connected k-sets (ESU)."""
    rp, col = _csr(g)
    lib = _load()
    return _hist_call(lib.oracle_count, g.n, _p(rp, ctypes.c_int32), _p(col, ctypes.c_int32), k,
                      nthreads or default_threads())


def count_roots(g, k: int, roots, nthreads: int | None = None):
    """Histogram of the connected k-sets whose smallest vertex is in ``roots``."""
    rp, col = _csr(g)
    roots = np.ascontiguousarray(roots, dtype=np.int32)
    lib = _load()
    return _hist_call(lib.oracle_count_roots, g.n, _p(rp, ctypes.c_int32),
                      _p(col, ctypes.c_int32), k, _p(roots, ctypes.c_int32), roots.size,
                      nthreads or default_threads())


def count_roots_split(g, k: int, roots, nthreads: int | None = None):
    """count_roots with each root's first-level extension steps spread over the
    threads (for hub roots, whose sets one thread would take minutes to list)."""
    rp, col = _csr(g)
    roots = np.ascontiguousarray(roots, dtype=np.int32)
    lib = _load()
    return _hist_call(lib.oracle_count_roots_split, g.n, _p(rp, ctypes.c_int32),
                      _p(col, ctypes.c_int32), k, _p(roots, ctypes.c_int32), roots.size,
                      nthreads or default_threads())


def count_bruteforce(g, k: int):
    """H_k(G) by trying every k-subset (n <= 64)."""
    rp, col = _csr(g)
    lib = _load()
    return _hist_call(lib.oracle_count_bruteforce, g.n, _p(rp, ctypes.c_int32),
                      _p(col, ctypes.c_int32), k)


def count_connected_sets(g, k: int, nthreads: int | None = None) -> int:
    rp, col = _csr(g)
    return int(_load().oracle_count_connected_sets(g.n, _p(rp, ctypes.c_int32),
                                                   _p(col, ctypes.c_int32), k,
                                                   nthreads or default_threads()))


def randomize(g, seed: int, swaps: int):
    """Sequential arc-swap null graph: returns (row_ptr, col, accepted swaps)."""
    rp, col = _csr(g)
    rp_out = np.empty(g.n + 1, np.int32)
    col_out = np.empty(max(g.m, 1), np.int32)
    acc = _load().oracle_randomize(g.n, _p(rp, ctypes.c_int32), _p(col, ctypes.c_int32), seed,
                                   swaps, _p(rp_out, ctypes.c_int32), _p(col_out, ctypes.c_int32))
    return rp_out, col_out[:g.m].copy(), int(acc)


def randomize_dyads(g, seed: int, attempts: int):
    """Dyad-preserving null graph: returns (row_ptr, col, accepted swaps)."""
    rp, col = _csr(g)
    rp_out = np.empty(g.n + 1, np.int32)
    col_out = np.empty(max(g.m, 1), np.int32)
    acc = _load().oracle_randomize_dyads(g.n, _p(rp, ctypes.c_int32), _p(col, ctypes.c_int32),
                                         seed, attempts, _p(rp_out, ctypes.c_int32),
                                         _p(col_out, ctypes.c_int32))
    return rp_out, col_out[:g.m].copy(), int(acc)


def zscores(h0, nulls) -> np.ndarray:
    """Per-class z-score of the original histogram against R null histograms.

    Sec. 1 step (c) names significance against the random ensemble without a
    formula; the reading is z = (H(G) - mu) / sigma with mu the mean and sigma the
    population standard deviation (ddof 0) of the R null counts, all in float64:
    mu = float(sum of the integer counts) / R; var = (sum over r, in seed order, of
    (float(h_r) - mu)^2) / R; sigma = sqrt(var); if sigma == 0 the z-score is 0
    when H(G) == mu and +-inf otherwise.  Loops are written out so that the
    order of every floating-point operation is explicit.
    """
    h0 = np.asarray(h0, dtype=np.uint64)
    nulls = np.asarray(nulls, dtype=np.uint64)
    R, C = nulls.shape
    z = np.empty(C, dtype=np.float64)
    for c in range(C):
        s1 = 0
        for r in range(R):
            s1 += int(nulls[r, c])
        mu = float(s1) / float(R)
        acc = 0.0
        for r in range(R):
            d = float(int(nulls[r, c])) - mu
            acc = acc + d * d
        var = acc / float(R)
        sigma = float(np.sqrt(np.float64(var)))
        diff = float(int(h0[c])) - mu
        if sigma == 0.0:
            z[c] = 0.0 if diff == 0.0 else (np.inf if diff > 0 else -np.inf)
        else:
            z[c] = diff / sigma
    return z
