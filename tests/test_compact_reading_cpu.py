"""The factorisation behind the compact k = 6 table, checked with the oracle's
brute-force canonical forms (CPU): relabelling the first four vertices X of a
6-vertex key into the canonical order of X's own class, and the fifth and
sixth vertices' fields for X's vertices with it, leaves the class of the whole
graph unchanged; and the connected 4-vertex prefixes fall into 199 classes."""
import itertools

import numpy as np

import oracle
from gpu_helpers import ext_key_to_mask

K = 6
XLOW = 18  # key bits of the fifth and sixth vertices' words


def key_off(p):
    return K * (K - 1) - p * (p + 1)


def field(key, p, q):
    """Two bits of position p's word for position q (bit 0: q -> p, bit 1: p -> q)."""
    return (key >> (key_off(p) + 2 * q)) & 3


def with_field(key, p, q, v):
    sh = key_off(p) + 2 * q
    return (key & ~(3 << sh)) | (v << sh)


def relabel_prefix(key, sigma):
    """New position i of X holds old vertex sigma[i]; positions 4, 5 stay."""
    out = key & ((1 << XLOW) - 1)  # the two words; their fields for X are rewritten below
    for p in range(1, 4):  # X's own arcs
        for q in range(p):
            a, b = sigma[q], sigma[p]  # arc bits between old vertices a, b
            if a < b:
                f = field(key, b, a)          # bit 0: a -> b, bit 1: b -> a
                v = f                         # new q -> new p is old a -> old b
            else:
                f = field(key, a, b)          # bit 0: b -> a, bit 1: a -> b
                v = ((f & 1) << 1) | (f >> 1)
            out = with_field(out, p, q, v)
    for p in (4, 5):  # the two words' fields for X's vertices
        for i in range(4):
            out = with_field(out, p, i, field(key, p, sigma[i]))
    return out


def x_mask(key):
    """Canonical-layout 4-vertex mask of the prefix X."""
    m = int(ext_key_to_mask(K, np.array([key & ~((1 << XLOW) - 1)], np.uint64))[0])
    out = 0
    for i in range(4):
        for j in range(4):
            if i != j and (m >> oracle.bit_index(K, i, j)) & 1:
                out |= 1 << oracle.bit_index(4, i, j)
    return out


def canonical_order(key):
    """The ordering sigma of X with the smallest 4-vertex mask."""
    best, best_sigma = None, None
    for sigma in itertools.permutations(range(4)):
        m = x_mask(relabel_prefix(key, sigma))
        if best is None or m < best:
            best, best_sigma = m, sigma
    return best, best_sigma


def test_relabelling_the_prefix_keeps_the_class():
    rng = np.random.default_rng(11)
    keys = rng.integers(0, 1 << 30, size=400, dtype=np.uint64)
    kept = 0
    for key in (int(k) for k in keys):
        if not oracle.connected(4, x_mask(key)):
            continue
        _, sigma = canonical_order(key)
        moved = relabel_prefix(key, sigma)
        a, b = ext_key_to_mask(K, np.array([key, moved], np.uint64))
        assert oracle.canon(K, int(a)) == oracle.canon(K, int(b))
        assert x_mask(moved) == oracle.canon(4, x_mask(key))
        kept += 1
    assert kept > 100


def test_connected_prefixes_have_199_classes():
    classes = {oracle.canon(4, x_mask(xk << XLOW)) for xk in range(1 << 12)
               if oracle.connected(4, x_mask(xk << XLOW))}
    assert len(classes) == 199
