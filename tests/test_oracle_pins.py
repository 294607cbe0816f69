"""Pins of the oracle against things other than itself: closed forms, brute force,
a library routine (networkx's triad census), the paper's worked example and
printed class counts, and metamorphic relations.  CPU only."""
import itertools
import json
import os
from math import comb

import numpy as np
import pytest

import oracle
import synthetic as syn
from closed_forms import connected_classes, digraph_classes, labelled_connected

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ------------------------------------------------------------------ canonical forms


def test_bit_layout_is_row_major_without_diagonal():
    for k in range(2, 7):
        seen = []
        for i in range(k):
            for j in range(k):
                if i != j:
                    seen.append(oracle.bit_index(k, i, j))
        assert seen == list(range(k * (k - 1)))


def test_closed_form_class_counts_match_paper():
    paper = _golden("paper_class_counts.json")
    cc = connected_classes(7)
    for k in ("3", "4", "5", "7"):
        assert cc[int(k)] == paper["paper"][k]
    # k = 6: the closed form gives one more class than the paper prints.
    assert cc[6] == paper["connected_closed_form"]["6"] == paper["paper"]["6"] + 1
    assert [digraph_classes(n) for n in range(1, 7)] == [1, 3, 16, 218, 9608, 1540944]


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_oracle_class_lists_match_closed_forms(k):
    conn = oracle.class_masks(k, True)
    allc = oracle.class_masks(k, False)
    assert len(conn) == connected_classes(k)[k]
    assert len(allc) == digraph_classes(k)
    assert np.all(np.diff(conn.astype(np.int64)) > 0)
    assert set(conn.tolist()) <= set(allc.tolist())


@pytest.mark.parametrize("k", [2, 3, 4])
def test_canon_partition_brute_force(k):
    """Every mask: orbit sizes divide k!, orbits partition the mask space, the
    connected masks number c(k) (labelled recurrence), canon is idempotent."""
    nb = k * (k - 1)
    masks = np.arange(1 << nb, dtype=np.uint32)
    can = oracle.canon_many(k, masks)
    assert np.all(can <= masks)
    assert np.array_equal(oracle.canon_many(k, can), can)
    vals, sizes = np.unique(can, return_counts=True)
    assert len(vals) == digraph_classes(k)
    assert all(__import__("math").factorial(k) % int(s) == 0 for s in sizes)
    nconn = sum(oracle.connected(k, int(m)) for m in masks)
    assert nconn == labelled_connected(k)[k]


def _relabel_mask(k, mask, perm):
    out = 0
    for i in range(k):
        for j in range(k):
            if i != j and (mask >> oracle.bit_index(k, i, j)) & 1:
                out |= 1 << oracle.bit_index(k, perm[i], perm[j])
    return out


@pytest.mark.parametrize("k", [5, 6])
def test_canon_invariant_under_relabelling(k):
    rng = np.random.default_rng(7)
    masks = rng.integers(0, 1 << (k * (k - 1)), size=200, dtype=np.uint64).astype(np.uint32)
    base = oracle.canon_many(k, masks)
    for t in range(3):
        perm = rng.permutation(k).tolist()
        moved = np.array([_relabel_mask(k, int(m), perm) for m in masks], dtype=np.uint32)
        assert np.array_equal(oracle.canon_many(k, moved), base)
    assert np.all(base <= masks)


def test_labelled_connected_counts_closed_form():
    assert labelled_connected(6)[1:] == [1, 3, 54, 3834, 1027080, 1067308488]


# ------------------------------------------------------------------ enumeration


def test_fig3_worked_example():
    fx = _golden("fig3_example.json")
    n = fx["n"]
    for orient in range(1 << len(fx["undirected_edges"])):
        src, dst = [], []
        for b, (u, v) in enumerate(fx["undirected_edges"]):
            if (orient >> b) & 1:
                src.append(u), dst.append(v)
            else:
                src.append(v), dst.append(u)
        g = syn.csr_from_arcs(n, src, dst)
        for r, sets in fx["connected_sets"].items():
            assert oracle.count_connected_sets(g, int(r)) == len(sets)
            _, nb = oracle.count_bruteforce(g, int(r))
            assert nb == len(sets)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_esu_equals_bruteforce_subsets(k, seed):
    n = [12, 16, 20, 24, 28, 30][seed]
    p = [0.35, 0.2, 0.12, 0.1, 0.08, 0.07][seed]
    if k == 6:
        n = min(n, 18)
    g = syn.random_small_digraph(n, p, 0.3, seed)
    h_esu, s_esu = oracle.count(g, k)
    h_bf, s_bf = oracle.count_bruteforce(g, k)
    assert s_esu == s_bf
    assert h_esu == h_bf
    assert sum(h_esu.values()) == s_esu
    # the same enumeration with each root's first-level steps spread over threads
    h_sp, s_sp = oracle.count_roots_split(g, k, np.arange(g.n), nthreads=3)
    assert (h_sp, s_sp) == (h_bf, s_bf)


def _triad_code_of_mask():
    nx = pytest.importorskip("networkx")
    codes = {}
    for mask in range(64):
        G = nx.DiGraph()
        G.add_nodes_from(range(3))
        for i in range(3):
            for j in range(3):
                if i != j and (mask >> oracle.bit_index(3, i, j)) & 1:
                    G.add_edge(i, j)
        census = nx.triadic_census(G)
        (code,) = [c for c, v in census.items() if v == 1]
        codes[mask] = code
    return codes


def test_k3_matches_networkx_triadic_census():
    nx = pytest.importorskip("networkx")
    codes = _triad_code_of_mask()
    classes = oracle.class_masks(3, True)
    class_codes = [codes[int(m)] for m in classes]
    assert len(set(class_codes)) == 13
    assert not set(class_codes) & {"003", "012", "102"}
    for seed in range(3):
        g = syn.uniform_digraph(60, 240 + 80 * seed, seed)
        h, _ = oracle.count(g, 3)
        G = nx.DiGraph()
        G.add_nodes_from(range(g.n))
        s, d = g.arcs()
        G.add_edges_from(zip(s.tolist(), d.tolist()))
        census = nx.triadic_census(G)
        for mask, cnt in h.items():
            assert census[codes[mask]] == cnt
        for code, cnt in census.items():
            if code not in ("003", "012", "102"):
                assert cnt == h.get(classes[class_codes.index(code)], 0)


def _canon_of_arcs(k, arcs):
    m = 0
    for i, j in arcs:
        m |= 1 << oracle.bit_index(k, i, j)
    return oracle.canon(k, m)


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_closed_form_families(k):
    n = 8
    full = (1 << (k * (k - 1))) - 1
    assert oracle.count(syn.complete_digraph(n), k)[0] == {full: comb(n, k)}
    assert oracle.count(syn.empty_graph(n), k) == ({}, 0)
    dpath = _canon_of_arcs(k, [(i, i + 1) for i in range(k - 1)])
    assert oracle.count(syn.directed_cycle(11), k)[0] == {dpath: 11}
    bip = _canon_of_arcs(k, [(i, i + 1) for i in range(k - 1)] + [(i + 1, i) for i in range(k - 1)])
    assert oracle.count(syn.bidirected_path(11), k)[0] == {bip: 11 - k + 1}
    star = _canon_of_arcs(k, [(0, i) for i in range(1, k)])
    assert oracle.count(syn.out_star(9), k)[0] == {star: comb(8, k - 1)}


def test_k3_total_closed_form():
    g = syn.chung_lu_digraph(400, 1600, 2.3, 60, 0.2, 3)
    s, d = g.arcs()
    und = {(min(a, b), max(a, b)) for a, b in zip(s.tolist(), d.tolist())}
    nbr = [set() for _ in range(g.n)]
    for a, b in und:
        nbr[a].add(b)
        nbr[b].add(a)
    tri = sum(len(nbr[a] & nbr[b]) for a, b in und) // 3
    expect = sum(comb(len(x), 2) for x in nbr) - 2 * tri
    h, sets = oracle.count(g, 3)
    assert sets == expect == sum(h.values())


def _transpose_mask(k, mask):
    out = 0
    for i in range(k):
        for j in range(k):
            if i != j and (mask >> oracle.bit_index(k, i, j)) & 1:
                out |= 1 << oracle.bit_index(k, j, i)
    return out


@pytest.mark.parametrize("k", [3, 4, 5])
def test_metamorphic_relations(k):
    g1 = syn.chung_lu_digraph(70, 220, 2.3, 20, 0.2, 11)
    g2 = syn.uniform_digraph(50, 160, 12)
    h1, s1 = oracle.count(g1, k)
    h2, _ = oracle.count(g2, k)
    # relabelling
    perm = np.random.default_rng(5).permutation(g1.n)
    assert oracle.count(syn.relabel(g1, perm), k)[0] == h1
    # disjoint union adds histograms
    hu, _ = oracle.count(syn.disjoint_union(g1, g2), k)
    want = dict(h1)
    for c, v in h2.items():
        want[c] = want.get(c, 0) + v
    assert hu == want
    # reversing all arcs maps every class to its transpose class
    hr, sr = oracle.count(syn.reverse(g1), k)
    assert sr == s1
    mapped = {oracle.canon(k, _transpose_mask(k, c)): v for c, v in h1.items()}
    assert hr == mapped


def test_split_roots_match_on_a_hub_graph():
    """A star with a few extra arcs: every set goes through one root's many
    first-level steps; the split count equals the closed form and the plain one."""
    from math import comb
    d = 40
    g = syn.out_star(d + 1)
    for k in (3, 4, 5):
        h, s = oracle.count_roots_split(g, k, np.arange(g.n), nthreads=4)
        assert s == comb(d, k - 1) and len(h) == 1
        assert (h, s) == oracle.count_roots(g, k, np.arange(g.n))


def test_count_roots_partitions_the_histogram():
    g = syn.chung_lu_digraph(120, 420, 2.3, 30, 0.1, 4)
    h, s = oracle.count(g, 4)
    ha, sa = oracle.count_roots(g, 4, np.arange(0, 50))
    hb, sb = oracle.count_roots(g, 4, np.arange(50, g.n))
    assert sa + sb == s
    merged = dict(ha)
    for c, v in hb.items():
        merged[c] = merged.get(c, 0) + v
    assert merged == h


# ------------------------------------------------------------------ randomiser


def test_splitmix64_published_vectors():
    fx = _golden("splitmix64_vectors.json")
    for i, hx in enumerate(fx["outputs_hex"]):
        assert oracle.splitmix64(fx["seed"], i) == int(hx, 16)


def test_randomize_hand_worked_swap():
    # Arcs (0->1), (2->3), seed 0, one attempt.  Outputs 0 and 1 of seed 0 have
    # top bits 1 and 0, so e1 = 1, e2 = 0: (a->b) = (2->3), (c->d) = (0->1); the
    # proposal (2->1), (0->3) passes every check and is accepted.
    g = syn.csr_from_arcs(4, [0, 2], [1, 3])
    rp, col, acc = oracle.randomize(g, 0, 1)
    assert acc == 1
    assert rp.tolist() == [0, 1, 1, 2, 2] and col.tolist() == [3, 1]
    # A 2-cycle can never swap (a == d on every proposal).
    g2 = syn.csr_from_arcs(2, [0, 1], [1, 0])
    rp2, col2, acc2 = oracle.randomize(g2, 9, 50)
    assert acc2 == 0 and col2.tolist() == [1, 0]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_randomize_invariants(seed):
    g = syn.chung_lu_digraph(300, 1200, 2.2, None, 0.1, 0)
    rp, col, acc = oracle.randomize(g, seed, 10 * g.m)
    assert acc > g.m  # most arcs moved
    assert np.array_equal(rp, g.row_ptr)  # out-degrees kept
    indeg0 = np.bincount(g.col, minlength=g.n)
    assert np.array_equal(np.bincount(col, minlength=g.n), indeg0)  # in-degrees kept
    src = np.repeat(np.arange(g.n), np.diff(rp))
    assert not np.any(src == col)  # no self-loops
    assert len(set(zip(src.tolist(), col.tolist()))) == g.m  # no duplicates
    for v in range(g.n):  # rows sorted
        assert np.all(np.diff(col[rp[v]:rp[v + 1]]) > 0)
    rp2, col2, acc2 = oracle.randomize(g, seed, 10 * g.m)
    assert acc2 == acc and np.array_equal(col2, col)
    _, col3, _ = oracle.randomize(g, seed + 100, 10 * g.m)
    assert not np.array_equal(col3, col)


# ------------------------------------------------------------------ z-scores


def test_zscores_closed_form_and_numpy():
    z = oracle.zscores([4, 2, 7], [[1, 2, 7], [3, 2, 7]])
    assert z[0] == 2.0 and z[1] == 0.0 and z[2] == 0.0
    z2 = oracle.zscores([5], [[2], [2]])
    assert z2[0] == np.inf
    rng = np.random.default_rng(0)
    nulls = rng.integers(0, 10**9, size=(64, 50), dtype=np.uint64)
    h0 = rng.integers(0, 10**9, size=50, dtype=np.uint64)
    z = oracle.zscores(h0, nulls)
    ref = (h0.astype(np.float64) - nulls.astype(np.float64).mean(0)) / nulls.astype(
        np.float64).std(0, ddof=0)
    np.testing.assert_allclose(z, ref, rtol=1e-12)


# ------------------------------------------------------------------ dyad-preserving randomiser


def _dyad_census(rp, col, n):
    src = np.repeat(np.arange(n), np.diff(rp))
    arcs = set(zip(src.tolist(), col.tolist()))
    mutual = {(a, b) for a, b in arcs if (b, a) in arcs and a < b}
    mdeg = np.zeros(n, int)
    for a, b in mutual:
        mdeg[a] += 1
        mdeg[b] += 1
    return len(mutual), len(arcs) - 2 * len(mutual), mdeg


def test_randomize_dyads_hand_worked_swap():
    # Two mutual dyads {0,1}, {2,3}: an attempt whose two picks differ (index =
    # top bit of outputs 1 and 2 of the seed, the kind pick is always "dyad")
    # turns them into {0,3}, {1,2}; equal picks leave the graph alone.
    g = syn.csr_from_arcs(4, [0, 1, 2, 3], [1, 0, 3, 2])
    for seed in range(40):
        i1 = oracle.splitmix64(seed, 1) >> 63
        i2 = oracle.splitmix64(seed, 2) >> 63
        rp, col, acc = oracle.randomize_dyads(g, seed, 1)
        if i1 != i2:
            assert acc == 1 and rp.tolist() == [0, 1, 2, 3, 4] and col.tolist() == [3, 2, 1, 0]
        else:
            assert acc == 0 and col.tolist() == [1, 0, 3, 2]


@pytest.mark.parametrize("seed", [1, 2])
def test_randomize_dyads_invariants(seed):
    g = syn.chung_lu_digraph(300, 1200, 2.2, None, 0.3, 0)
    rp, col, acc = oracle.randomize_dyads(g, seed, 10 * g.m)
    assert acc > g.m // 2
    assert np.array_equal(rp, g.row_ptr)  # out-degrees
    assert np.array_equal(np.bincount(col, minlength=g.n), np.bincount(g.col, minlength=g.n))
    src = np.repeat(np.arange(g.n), np.diff(rp))
    assert not np.any(src == col) and len(set(zip(src.tolist(), col.tolist()))) == g.m
    m0, s0, d0 = _dyad_census(g.row_ptr, g.col, g.n)
    m1, s1, d1 = _dyad_census(rp, col, g.n)
    assert (m0, s0) == (m1, s1) and np.array_equal(d0, d1)  # reciprocity kept
    assert not np.array_equal(col, g.col)
    rp2, col2, acc2 = oracle.randomize_dyads(g, seed, 10 * g.m)
    assert acc2 == acc and np.array_equal(col2, col)
    # the plain arc swap does not keep the dyad census
    _, colp, _ = oracle.randomize(g, seed, 10 * g.m)
    assert _dyad_census(rp, colp, g.n)[0] != m0
