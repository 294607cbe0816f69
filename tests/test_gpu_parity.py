"""Parity of the CUDA path with the oracle (bit-exact: all of this is integer
work), through the C ABI.  GPU only."""
import numpy as np
import pytest

import oracle
import synthetic as syn
from closed_forms import connected_classes
from gpu_helpers import expected_ids, oracle_dense

pytestmark = pytest.mark.gpu

ORACLE_CLASSES = {}


def oracle_classes(k):
    if k not in ORACLE_CLASSES:
        ORACLE_CLASSES[k] = oracle.class_masks(k) if k <= 5 else None
    return ORACLE_CLASSES[k]


@pytest.fixture(scope="session")
def tables(lib):
    lib.load_library()
    out = {}

    def get(k):
        if k not in out:
            out[k] = lib.table_build(k)
        return out[k]
    return get


def gpu_hist(lib, t, g, via="host", method=0):
    dg = lib.graph_from(g)
    if method:
        h = lib.to_numpy_u64(lib.count_tuned(dg, t, method=method))
        assert lib.count_stats(dg)[1] == 0
    elif via == "host":
        h = lib.count_host(dg, t)
    else:
        h = lib.to_numpy_u64(lib.count(dg, t))
        items, err, ms = lib.count_stats(dg)
        assert err == 0
    return h, dg


METHODS = [0, 1]  # per-subgraph classification, cell-pair counting


def check_against_oracle(lib, t, g, k, via="host", method=0):
    h, _ = gpu_hist(lib, t, g, via, method)
    want, sets = oracle.count(g, k)
    assert int(h.sum()) == sets
    np.testing.assert_array_equal(h, oracle_dense(want, t.class_masks()))


# ------------------------------------------------------------------ table (K1)


@pytest.mark.parametrize("k", [3, 4, 5])
def test_table_every_key_matches_oracle(lib, tables, k):
    t = tables(k)
    cm = oracle_classes(k)
    assert t.num_classes == len(cm) == connected_classes(k)[k]
    np.testing.assert_array_equal(t.class_masks(), cm)
    nkeys = 1 << (k * (k - 1))
    keys = np.arange(nkeys, dtype=np.uint64)
    np.testing.assert_array_equal(t.entries(0, nkeys), expected_ids(k, keys, cm))


def test_table_k6_classes_and_sampled_keys(lib, tables):
    t = tables(6)
    cm = t.class_masks()
    assert t.num_classes == len(cm) == connected_classes(6)[6] == 1530843
    assert np.all(np.diff(cm.astype(np.int64)) > 0)
    rng = np.random.default_rng(1)
    # every class mask is the oracle's canonical form of itself and connected
    np.testing.assert_array_equal(oracle.canon_many(6, cm), cm)
    assert all(oracle.connected(6, int(m)) for m in cm)
    # random keys and keys of sparse patterns (few arcs), as the enumerator sees them
    keys = rng.integers(0, 1 << 30, size=80000, dtype=np.uint64)
    sparse = np.zeros(40000, np.uint64)
    for b in range(6):
        sparse |= np.uint64(1) << rng.integers(0, 30, size=40000).astype(np.uint64)
    keys = np.concatenate([keys, sparse])
    got = np.array([t.entries(int(x), 1)[0] for x in keys[:2000]], np.uint32)
    want = expected_ids(6, keys, cm)
    np.testing.assert_array_equal(got, want[:2000])
    # bulk: read the slots in ranges around the sampled keys
    order = np.argsort(keys)
    ks = keys[order]
    block = t.entries(0, 1 << 22)  # the first 4M slots in one read
    inblk = ks < (1 << 22)
    np.testing.assert_array_equal(block[ks[inblk].astype(np.int64)], want[order][inblk])


def test_table_k6_ten_million_random_keys(lib, tables):
    """10^7 random 6-vertex keys: the table's class id equals the oracle's
    (brute-force canonical form over the 720 orderings, ranked among the class
    masks), read back in 64 MB slices of the 4 GiB table."""
    t = tables(6)
    cm = t.class_masks()
    rng = np.random.default_rng(7)
    keys = np.unique(rng.integers(0, 1 << 30, size=10_000_000, dtype=np.uint64))
    want = expected_ids(6, keys, cm)
    got = np.empty(keys.size, np.uint32)
    span = 1 << 24
    starts = np.searchsorted(keys, np.arange(0, (1 << 30) + 1, span, dtype=np.uint64))
    for i in range((1 << 30) // span):
        a, b = starts[i], starts[i + 1]
        if a == b:
            continue
        block = t.entries(i * span, span)
        got[a:b] = block[(keys[a:b] - np.uint64(i * span)).astype(np.int64)]
    np.testing.assert_array_equal(got, want)


# ------------------------------------------------------------------ counting (K2)


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("k", [3, 4, 5, 6])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_small_random_digraphs(lib, tables, k, seed, method):
    n = [14, 22, 30][seed]
    g = syn.random_small_digraph(n, [0.3, 0.15, 0.1][seed], 0.3, seed)
    check_against_oracle(lib, tables(k), g, k, via="host" if seed % 2 else "device",
                         method=method)


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_closed_form_families_and_edges(lib, tables, k, method):
    t = tables(k)
    for g in [syn.complete_digraph(9), syn.directed_cycle(13), syn.bidirected_path(12),
              syn.out_star(40), syn.empty_graph(10), syn.empty_graph(1), syn.complete_digraph(k - 1),
              syn.reverse(syn.out_star(33)),
              syn.disjoint_union(syn.complete_digraph(7), syn.empty_graph(5))]:
        check_against_oracle(lib, t, g, k, method=method)


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_medium_power_law_graphs(lib, tables, k, method):
    # several tiles per row and ragged tails: hubs of degree ~60-100
    n, m = {3: (900, 4000), 4: (600, 2400), 5: (300, 1000), 6: (160, 420)}[k]
    g = syn.chung_lu_digraph(n, m, 2.2, None, 0.15, 10 + k)
    check_against_oracle(lib, tables(k), g, k, method=method)


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("k", [4, 5, 6])
def test_large_graph_relation_words_in_global_memory(lib, tables, k, method):
    """n = 20,000: one warp's relation words (n bytes, 2n at k = 6) cannot sit
    in shared memory beside 16 warps' stacks, so the launch keeps them in
    global memory, one 16-byte-aligned slice per warp (the k = 5 enumerator
    updates them with 32-bit atomics).  k = 4, 5 against the whole oracle
    histogram; k = 6 on root ranges away from the hubs, plus the property that
    disjoint ranges add up to the whole count (of either method)."""
    g = syn.chung_lu_digraph(20000, 24000, 2.5, 30, 0.1, 77)
    t = tables(k)
    if k <= 5:
        check_against_oracle(lib, t, g, k, method=method)
        return
    dg = lib.graph_from(g)
    cm = t.class_masks()
    for a, b in [(800, 850), (1500, 1600), (3000, 3200)]:
        want, sets = oracle.count_roots(g, 6, np.arange(a, b))
        h = lib.count_roots(dg, t, a, b)
        assert int(h.sum()) == sets
        np.testing.assert_array_equal(h, oracle_dense(want, cm))
    full = lib.to_numpy_u64(lib.count_tuned(dg, t, method=method))
    assert lib.count_stats(dg)[1] == 0
    parts = sum(lib.count_roots(dg, t, a, b) for a, b in [(0, 800), (800, 850), (850, 20000)])
    np.testing.assert_array_equal(parts, full)


@pytest.mark.parametrize("k", [3, 4, 5, 6])
@pytest.mark.parametrize("split", [1.0, 1e12])
@pytest.mark.parametrize("wpb", [1, 16])
def test_cells_work_splitting_is_exact(lib, tables, k, split, wpb):
    """The cell method under every split (k = 4 splits exactly at its pair level)."""
    n, m = {3: (400, 1500), 4: (300, 1100), 5: (150, 450), 6: (90, 220)}[k]
    g = syn.chung_lu_digraph(n, m, 2.1, None, 0.2, 78)
    t = tables(k)
    dg = lib.graph_from(g)
    h = lib.to_numpy_u64(lib.count_tuned(dg, t, split, wpb, method=1))
    assert lib.count_stats(dg)[1] == 0
    np.testing.assert_array_equal(h, oracle_dense(oracle.count(g, k)[0], t.class_masks()))


@pytest.mark.parametrize("k", [4, 5, 6])
@pytest.mark.parametrize("split", [1.0, 50.0, 1e12])
@pytest.mark.parametrize("wpb", [1, 4, 16])
def test_work_splitting_is_exact(lib, tables, k, split, wpb):
    """Every split of the work (all first branches split into second-level
    items, a mix, none) and every block size gives the oracle's histogram."""
    n, m = {4: (300, 1100), 5: (150, 450), 6: (90, 220)}[k]
    g = syn.chung_lu_digraph(n, m, 2.1, None, 0.2, 77)
    t = tables(k)
    dg = lib.graph_from(g)
    h = lib.to_numpy_u64(lib.count_tuned(dg, t, split, wpb))
    items, err, _ = lib.count_stats(dg)
    assert err == 0 and items > 0
    want, sets = oracle.count(g, k)
    np.testing.assert_array_equal(h, oracle_dense(want, t.class_masks()))


@pytest.mark.parametrize("method", METHODS)
def test_workload_uniform_k3_full(lib, tables, method):
    g = syn.workload_graph("uniform_k3")
    check_against_oracle(lib, tables(3), g, 3, via="device", method=method)


@pytest.mark.parametrize("method", METHODS)
def test_workload_chunglu_k4_full(lib, tables, method):
    g = syn.workload_graph("chunglu_k4")
    check_against_oracle(lib, tables(4), g, 4, via="device", method=method)


SAMPLES = {
    # root ranges the oracle finishes in seconds; they include mid-degree roots
    "nullmodel_k5": [(500, 520), (200, 205), (50, 52), (1000, 1500)],
    "nullmodel_k6": [(400, 420), (200, 205), (50, 52), (600, 800)],
}


@pytest.mark.parametrize("name", ["nullmodel_k5", "nullmodel_k6"])
def test_full_size_root_samples_and_partition(lib, tables, name):
    k = syn.WORKLOADS[name]["k"]
    g = syn.workload_graph(name)
    t = tables(k)
    dg = lib.graph_from(g)
    cm = t.class_masks()
    for a, b in SAMPLES[name]:
        h = lib.count_roots(dg, t, a, b)
        want, sets = oracle.count_roots(g, k, np.arange(a, b))
        assert int(h.sum()) == sets
        np.testing.assert_array_equal(h, oracle_dense(want, cm))
    # property at full size: disjoint root ranges add up to the whole count,
    # and the whole count does not depend on how the work is split
    full = lib.to_numpy_u64(lib.count(dg, t))
    cuts = [0, 1, 2, 5, 17, 64, 300, g.n]
    parts = sum(lib.count_roots(dg, t, cuts[i], cuts[i + 1]) for i in range(len(cuts) - 1))
    np.testing.assert_array_equal(parts, full)
    nosplit = lib.to_numpy_u64(lib.count_tuned(dg, t, 1e15, 8))
    np.testing.assert_array_equal(nosplit, full)
    assert lib.count_stats(dg)[1] == 0
    # the cell method counts the same histogram at full size
    cells = lib.to_numpy_u64(lib.count_tuned(dg, t, method=1))
    assert lib.count_stats(dg)[1] == 0
    np.testing.assert_array_equal(cells, full)


def test_largest_graph_the_loader_takes(lib, tables):
    """n = 65,535, the most vertices a graph may have (ids are 16 bits in the
    candidate stacks and in the randomiser's arc keys), relabelled so that the
    hubs carry the highest ids: the whole k = 3 histogram and a k = 4 root
    range against the oracle, and a null graph bit for bit."""
    g0 = syn.chung_lu_digraph(65535, 130000, 2.5, 60, 0.15, 99)
    g = syn.relabel(g0, np.arange(g0.n)[::-1])
    dg = lib.graph_from(g)
    assert dg.n == 65535
    check_against_oracle(lib, tables(3), g, 3, via="device")
    t4 = tables(4)
    h = lib.count_roots(dg, t4, 30000, 30400)
    want, sets = oracle.count_roots(g, 4, np.arange(30000, 30400))
    assert sets > 0 and int(h.sum()) == sets
    np.testing.assert_array_equal(h, oracle_dense(want, t4.class_masks()))
    r = lib.randomize(dg, 5, 10 * g.m)
    rp, col = r.copy_csr()
    orp, ocol, _ = oracle.randomize(g, 5, 10 * g.m)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(col, ocol)


def test_k5_workload_whole_graph_vs_oracle(lib, tables):
    """The whole k = 5 workload graph, hub roots included (the roots the
    enumerator splits into second-level items and donates between warps),
    against the oracle, whose hub roots are spread over the host's threads
    branch by branch (about 8e8 sets)."""
    g = syn.workload_graph("nullmodel_k5")
    t = tables(5)
    dg = lib.graph_from(g)
    h = lib.to_numpy_u64(lib.count(dg, t))
    assert lib.count_stats(dg)[1] == 0
    want, sets = oracle.count_roots_split(g, 5, np.arange(g.n))
    assert int(h.sum()) == sets
    np.testing.assert_array_equal(h, oracle_dense(want, t.class_masks()))


def test_k6_workload_hub_roots_vs_oracle(lib, tables):
    """The two largest hubs of the k = 6 workload graph (roots 0 and 1, about
    5e7 sets), against the oracle."""
    g = syn.workload_graph("nullmodel_k6")
    t = tables(6)
    dg = lib.graph_from(g)
    h = lib.count_roots(dg, t, 0, 2)
    want, sets = oracle.count_roots_split(g, 6, np.arange(0, 2))
    assert int(h.sum()) == sets
    np.testing.assert_array_equal(h, oracle_dense(want, t.class_masks()))


# ------------------------------------------------------------------ randomiser (K3)


@pytest.mark.parametrize("name,seeds", [("nullmodel_k5", [1, 2, 3]), ("nullmodel_k6", [1, 64]),
                                        ("chunglu_k4", [5])])
def test_randomize_bit_exact(lib, name, seeds):
    g = syn.workload_graph(name)
    dg = lib.graph_from(g)
    for s in seeds:
        r = lib.randomize(dg, s, 10 * g.m)
        rp, col = r.copy_csr()
        orp, ocol, acc = oracle.randomize(g, s, 10 * g.m)
        np.testing.assert_array_equal(rp, orp)
        np.testing.assert_array_equal(col, ocol)
        assert acc > 0


def test_randomize_small_edge_cases(lib):
    for g, swaps in [(syn.csr_from_arcs(4, [0, 2], [1, 3]), 1), (syn.directed_cycle(3), 100),
                     (syn.complete_digraph(5), 50), (syn.empty_graph(3), 10),
                     (syn.random_small_digraph(30, 0.2, 0.3, 4), 0),
                     (syn.random_small_digraph(30, 0.2, 0.3, 4), 997)]:
        dg = lib.graph_from(g)
        r = lib.randomize(dg, 0, swaps)
        rp, col = r.copy_csr()
        orp, ocol, _ = oracle.randomize(g, 0, swaps)
        np.testing.assert_array_equal(rp, orp)
        np.testing.assert_array_equal(col, ocol)


@pytest.mark.parametrize("name,seeds", [("nullmodel_k5", [1, 2]), ("nullmodel_k6", [3]),
                                        ("chunglu_k4", [4])])
def test_randomize_dyads_bit_exact(lib, name, seeds):
    g = syn.workload_graph(name)
    dg = lib.graph_from(g)
    for s in seeds:
        r = lib.randomize_dyads(dg, s, 10 * g.m)
        rp, col = r.copy_csr()
        orp, ocol, acc = oracle.randomize_dyads(g, s, 10 * g.m)
        np.testing.assert_array_equal(rp, orp)
        np.testing.assert_array_equal(col, ocol)
        assert acc > 0


def test_randomize_dyads_small_cases(lib):
    for g, att in [(syn.csr_from_arcs(4, [0, 1, 2, 3], [1, 0, 3, 2]), 1),
                   (syn.complete_digraph(5), 40), (syn.empty_graph(3), 5),
                   (syn.random_small_digraph(40, 0.15, 0.5, 9), 0),
                   (syn.random_small_digraph(40, 0.15, 0.5, 9), 2000),
                   (syn.directed_cycle(9), 300)]:
        for seed in (0, 5):
            r = lib.randomize_dyads(lib.graph_from(g), seed, att)
            rp, col = r.copy_csr()
            orp, ocol, _ = oracle.randomize_dyads(g, seed, att)
            np.testing.assert_array_equal(rp, orp)
            np.testing.assert_array_equal(col, ocol)


@pytest.mark.parametrize("model", ["arcs", "dyads"])
def test_randomize_large_graph_state_in_global_memory(lib, model):
    """m = 50,000: the arc set does not fit shared memory, so the randomiser
    keeps it in global memory; the null graph is still bit-exact (both null
    models; the dyad one refused such graphs before)."""
    g = syn.chung_lu_digraph(20000, 50000, 2.4, 200, 0.2, 21)
    dg = lib.graph_from(g)
    fn, ofn = ((lib.randomize, oracle.randomize) if model == "arcs"
               else (lib.randomize_dyads, oracle.randomize_dyads))
    r = fn(dg, 9, 10 * g.m)
    rp, col = r.copy_csr()
    orp, ocol, acc = ofn(g, 9, 10 * g.m)
    assert acc > 0
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(col, ocol)


def test_randomize_dense_graphs(lib):
    """Complete and near-complete digraphs (most attempts rejected, buckets
    full of structured keys), both null models, against the oracle."""
    for g in [syn.complete_digraph(40), syn.random_small_digraph(60, 0.6, 0.5, 3)]:
        dg = lib.graph_from(g)
        for fn, ofn in [(lib.randomize, oracle.randomize),
                        (lib.randomize_dyads, oracle.randomize_dyads)]:
            r = fn(dg, 4, 10 * g.m)
            rp, col = r.copy_csr()
            orp, ocol, _ = ofn(g, 4, 10 * g.m)
            np.testing.assert_array_equal(rp, orp)
            np.testing.assert_array_equal(col, ocol)


def test_duplicate_arc_rejected_on_device(lib):
    with pytest.raises(lib.MotifsError) as ei:
        lib.graph_load_csr(3, [0, 2, 2, 2], [1, 1])
    assert ei.value.status == lib.MT_EINVAL


# ------------------------------------------------------------------ batch (a7-a9) + z (K5)


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("k,n,m,R", [(4, 200, 700, 6), (5, 120, 380, 5), (6, 70, 180, 4),
                                     (3, 300, 1500, 9)])
def test_batch_small_vs_oracle(lib, tables, k, n, m, R, method):
    g = syn.chung_lu_digraph(n, m, 2.3, None, 0.1, 100 + k)
    t = tables(k)
    dg = lib.graph_from(g)
    seeds = np.arange(1, R + 1, dtype=np.uint64)
    b = lib.Batch(dg, t, R, 10 * g.m, lib.make_tuning(method=method) if method else None)
    for rep in range(2):  # second run replays the captured graph
        hists, z = b.run(seeds)
        hists = lib.to_numpy_u64(hists)
        z = z.cpu().numpy()
        assert b.error() == 0
        cm = t.class_masks()
        np.testing.assert_array_equal(hists[0], oracle_dense(oracle.count(g, k)[0], cm))
        for r in range(R):
            rp, col, _ = oracle.randomize(g, int(seeds[r]), 10 * g.m)
            gr = syn.Graph(g.n, rp, col)
            np.testing.assert_array_equal(hists[r + 1], oracle_dense(oracle.count(gr, k)[0], cm))
        zo = oracle.zscores(hists[0], hists[1:])
        np.testing.assert_array_equal(z, zo)  # same float64 operations in the same order
    if method:
        return
    # host buffers through the one-shot entry point
    h2, z2 = lib.count_batch(dg, t, seeds, 10 * g.m)
    np.testing.assert_array_equal(h2, hists)
    np.testing.assert_array_equal(z2, z)


def test_batch_full_size_k5(lib, tables):
    """The benchmark's launch configuration (original + 256 nulls, one launch):
    every row equals the one-graph count of the same null graph; null graphs
    are the oracle's bit for bit; rows are checked against the oracle on root
    samples; z equals the oracle's float64 formula on these counts."""
    name = "nullmodel_k5"
    g = syn.workload_graph(name)
    t = tables(5)
    dg = lib.graph_from(g)
    R = syn.WORKLOADS[name]["nulls"]
    seeds = np.arange(1, R + 1, dtype=np.uint64)
    b = lib.Batch(dg, t, R, 10 * g.m)
    hists, z = b.run(seeds)
    hists = lib.to_numpy_u64(hists)
    z = z.cpu().numpy()
    assert b.error() == 0
    np.testing.assert_array_equal(hists[0], lib.to_numpy_u64(lib.count(dg, t)))
    cm = t.class_masks()
    for r in [0, 1, 128, 255]:
        nul = lib.randomize(dg, int(seeds[r]), 10 * g.m)
        np.testing.assert_array_equal(hists[r + 1], lib.to_numpy_u64(lib.count(nul, t)))
        if r in (0, 255):
            rp, col, _ = oracle.randomize(g, int(seeds[r]), 10 * g.m)
            gr = syn.Graph(g.n, rp, col)
            np.testing.assert_array_equal(nul.copy_csr()[1], col)
            want, _ = oracle.count_roots(gr, 5, np.arange(500, 530))
            np.testing.assert_array_equal(lib.count_roots(nul, t, 500, 530), oracle_dense(want, cm))
    np.testing.assert_array_equal(z, oracle.zscores(hists[0], hists[1:]))


def test_batch_k6_many_graphs_vs_oracle(lib, tables):
    """k = 6 over 64 graphs: with few blocks per graph the enumerator groups a
    tail batch's leaves with one match for all choices (with many blocks per
    graph, three choices per match); every row against the oracle's count of
    the oracle's null graph."""
    g = syn.chung_lu_digraph(60, 120, 2.3, None, 0.1, 106)
    t = tables(6)
    dg = lib.graph_from(g)
    R = 63
    roots = np.arange(g.n)
    assert lib.launch_info(dg, 6)["blocks"] <= 3 * (R + 1)
    seeds = np.arange(1, R + 1, dtype=np.uint64)
    b = lib.Batch(dg, t, R, 10 * g.m)
    hists, z = b.run(seeds)
    hists = lib.to_numpy_u64(hists)
    assert b.error() == 0
    cm = t.class_masks()
    np.testing.assert_array_equal(hists[0], oracle_dense(oracle.count_roots_split(g, 6, roots)[0], cm))
    for r in range(R):
        rp, col, _ = oracle.randomize(g, int(seeds[r]), 10 * g.m)
        want, _ = oracle.count_roots_split(syn.Graph(g.n, rp, col), 6, roots)
        np.testing.assert_array_equal(hists[r + 1], oracle_dense(want, cm))
    np.testing.assert_array_equal(z.cpu().numpy(), oracle.zscores(hists[0], hists[1:]))


def test_batch_full_size_k6(lib, tables):
    """The k = 6 benchmark launch (original + 64 nulls, one launch, one match
    per tail batch): sampled rows equal one-graph counts of the same null
    graphs (launches of one graph, three choices per match) and the oracle on
    root samples."""
    name = "nullmodel_k6"
    g = syn.workload_graph(name)
    t = tables(6)
    dg = lib.graph_from(g)
    R = syn.WORKLOADS[name]["nulls"]
    info = lib.launch_info(dg, 6)
    assert 3 < info["blocks"] <= 3 * (R + 1)
    seeds = np.arange(1, R + 1, dtype=np.uint64)
    b = lib.Batch(dg, t, R, 10 * g.m)
    hists, z = b.run(seeds)
    hists = lib.to_numpy_u64(hists)
    assert b.error() == 0
    np.testing.assert_array_equal(hists[0], lib.to_numpy_u64(lib.count(dg, t)))
    cm = t.class_masks()
    for r in [0, 31, 63]:
        nul = lib.randomize(dg, int(seeds[r]), 10 * g.m)
        np.testing.assert_array_equal(hists[r + 1], lib.to_numpy_u64(lib.count(nul, t)))
        if r == 63:
            rp, col, _ = oracle.randomize(g, int(seeds[r]), 10 * g.m)
            np.testing.assert_array_equal(nul.copy_csr()[1], col)
            want, _ = oracle.count_roots(syn.Graph(g.n, rp, col), 6, np.arange(600, 640))
            np.testing.assert_array_equal(lib.count_roots(nul, t, 600, 640), oracle_dense(want, cm))
    np.testing.assert_array_equal(z.cpu().numpy(), oracle.zscores(hists[0], hists[1:]))


@pytest.mark.parametrize("method", METHODS)
def test_batch_dyad_null_model(lib, tables, method):
    """The batch with the dyad-preserving null model: rows equal the oracle's
    counts of the oracle's dyad-preserving null graphs; z from its formula."""
    g = syn.chung_lu_digraph(150, 500, 2.3, None, 0.3, 21)
    t = tables(4)
    dg = lib.graph_from(g)
    R = 5
    seeds = np.arange(1, R + 1, dtype=np.uint64)
    tun = lib.make_tuning(method=method) if method else None
    b = lib.Batch(dg, t, R, 10 * g.m, tun, null_model=lib.NULL_DYAD_SWAP)
    hists, z = b.run(seeds)
    hists = lib.to_numpy_u64(hists)
    assert b.error() == 0
    cm = t.class_masks()
    for r in range(R):
        rp, col, _ = oracle.randomize_dyads(g, int(seeds[r]), 10 * g.m)
        np.testing.assert_array_equal(hists[r + 1],
                                      oracle_dense(oracle.count(syn.Graph(g.n, rp, col), 4)[0], cm))
    np.testing.assert_array_equal(z.cpu().numpy(), oracle.zscores(hists[0], hists[1:]))

