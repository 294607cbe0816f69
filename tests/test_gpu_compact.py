"""The compact k = 6 table (mt_table_build_compact): its slots against the
oracle's canonical forms, and counts with it against the oracle and the full
table.  GPU only."""
import numpy as np
import pytest

import oracle
import synthetic as syn
from gpu_helpers import expected_ids, oracle_dense

pytestmark = pytest.mark.gpu

XLOW = 18  # bits of the fifth and sixth vertices' words in a 6-vertex key


@pytest.fixture(scope="module")
def tables(lib):
    lib.load_library()
    full = lib.table_build(6)
    compact = lib.table_build(6, compact=True)
    yield full, compact
    compact.free()
    full.free()


def xkey_of_mask4(mask4: int) -> int:
    """Key bits of positions 1..3 of a 6-vertex key (before the shift by 18)
    for the 4-vertex graph with canonical-layout mask `mask4`."""
    out = 0
    for p in range(1, 4):
        off = 6 * 5 - p * (p + 1) - XLOW
        for q in range(p):
            if (mask4 >> oracle.bit_index(4, q, p)) & 1:  # q -> p
                out |= 1 << (off + 2 * q)
            if (mask4 >> oracle.bit_index(4, p, q)) & 1:  # p -> q
                out |= 1 << (off + 2 * q + 1)
    return out


def test_compact_table_shape(tables):
    full, compact = tables
    assert compact.compact and not full.compact
    assert compact.num_classes == full.num_classes == 1530843
    np.testing.assert_array_equal(compact.class_masks(), full.class_masks())


def test_compact_slots_against_oracle(tables):
    """Slot (c, y, z) is the class of: the c-th connected 4-vertex canonical
    form (ascending canonical-layout masks, as the oracle lists them) as the
    first four vertices, y as the fifth vertex's word and z as the sixth's."""
    _, compact = tables
    reps = oracle.class_masks(4)
    assert len(reps) == 199
    rng = np.random.default_rng(3)
    slots = rng.integers(0, 199 << XLOW, size=4000, dtype=np.int64)
    # every class of X, a dense block at the start and the very last slot
    slots = np.concatenate([slots, (np.arange(199, dtype=np.int64) << XLOW) + 12345,
                            np.arange(2048, dtype=np.int64), [(199 << XLOW) - 1]])
    keys = np.array([(xkey_of_mask4(int(reps[s >> XLOW])) << XLOW) | (s & ((1 << XLOW) - 1))
                     for s in slots], dtype=np.uint64)
    want = expected_ids(6, keys, compact.class_masks())
    order = np.argsort(slots)
    got = np.empty(len(slots), np.uint32)
    # read in a few contiguous blocks
    for lo in range(0, 199 << XLOW, 1 << 22):
        sel = (slots[order] >= lo) & (slots[order] < lo + (1 << 22))
        if not sel.any():
            continue
        block = compact.entries(lo, min(1 << 22, (199 << XLOW) - lo))
        got[order[sel]] = block[slots[order][sel] - lo]
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_compact_counts_small_graphs(lib, tables, seed):
    full, compact = tables
    n = [14, 22, 30][seed]
    g = syn.random_small_digraph(n, [0.3, 0.15, 0.1][seed], 0.3, seed)
    dg = lib.graph_from(g)
    h = lib.count_host(dg, compact)
    want, sets = oracle.count(g, 6)
    assert int(h.sum()) == sets
    np.testing.assert_array_equal(h, oracle_dense(want, compact.class_masks()))
    np.testing.assert_array_equal(h, lib.count_host(dg, full))


def test_compact_counts_power_law_and_families(lib, tables):
    full, compact = tables
    graphs = [syn.chung_lu_digraph(160, 420, 2.2, None, 0.15, 16), syn.complete_digraph(9),
              syn.directed_cycle(13), syn.bidirected_path(12), syn.out_star(40),
              syn.reverse(syn.out_star(33)),
              syn.disjoint_union(syn.complete_digraph(7), syn.empty_graph(5))]
    for g in graphs:
        dg = lib.graph_from(g)
        h = lib.to_numpy_u64(lib.count(dg, compact))
        assert lib.count_stats(dg)[1] == 0
        want, sets = oracle.count(g, 6)
        assert int(h.sum()) == sets
        np.testing.assert_array_equal(h, oracle_dense(want, compact.class_masks()))
        np.testing.assert_array_equal(h, lib.count_host(dg, full))


def test_compact_full_size_workload(lib, tables):
    """The k = 6 workload graph: root samples against the oracle, the whole
    count against the full table's, and a small null-model batch."""
    full, compact = tables
    g = syn.workload_graph("nullmodel_k6")
    dg = lib.graph_from(g)
    cm = compact.class_masks()
    for a, b in [(400, 420), (50, 52)]:
        want, sets = oracle.count_roots(g, 6, np.arange(a, b))
        h = lib.count_roots(dg, compact, a, b)
        assert int(h.sum()) == sets
        np.testing.assert_array_equal(h, oracle_dense(want, cm))
    np.testing.assert_array_equal(lib.to_numpy_u64(lib.count(dg, compact)),
                                  lib.to_numpy_u64(lib.count(dg, full)))
    assert lib.count_stats(dg)[1] == 0
    seeds = np.arange(1, 5, dtype=np.uint64)
    bc = lib.Batch(dg, compact, 4, 10 * g.m)
    hc, zc = bc.run(seeds)
    hc, zc = lib.to_numpy_u64(hc), zc.cpu().numpy()
    assert bc.error() == 0
    bf = lib.Batch(dg, full, 4, 10 * g.m)
    hf, zf = bf.run(seeds)
    np.testing.assert_array_equal(hc, lib.to_numpy_u64(hf))
    np.testing.assert_array_equal(zc, zf.cpu().numpy())
    bc.free()
    bf.free()
    np.testing.assert_array_equal(lib.to_numpy_u64(lib.count_noalloc(dg, compact)),
                                  lib.to_numpy_u64(lib.count(dg, full)))


def test_compact_batch_many_graphs(lib, tables):
    """64 graphs in one launch (at most 3 blocks per graph: one match per tail
    batch) with the compact table: rows equal the full table's batch, sampled
    rows the oracle, and a few rows the one-graph counts (three choices per
    match) with the compact table."""
    full, compact = tables
    g = syn.chung_lu_digraph(60, 120, 2.3, None, 0.1, 106)
    dg = lib.graph_from(g)
    R = 63
    assert lib.launch_info(dg, 6)["blocks"] <= 3 * (R + 1)
    seeds = np.arange(1, R + 1, dtype=np.uint64)
    bc = lib.Batch(dg, compact, R, 10 * g.m)
    hc, zc = bc.run(seeds)
    hc, zc = lib.to_numpy_u64(hc), zc.cpu().numpy()
    assert bc.error() == 0
    bf = lib.Batch(dg, full, R, 10 * g.m)
    hf, zf = bf.run(seeds)
    np.testing.assert_array_equal(hc, lib.to_numpy_u64(hf))
    np.testing.assert_array_equal(zc, zf.cpu().numpy())
    bc.free()
    bf.free()
    cm = compact.class_masks()
    for r in (0, 17, 62):
        rp, col, _ = oracle.randomize(g, int(seeds[r]), 10 * g.m)
        gr = syn.Graph(g.n, rp, col)
        want, _ = oracle.count_roots_split(gr, 6, np.arange(g.n))
        np.testing.assert_array_equal(hc[r + 1], oracle_dense(want, cm))
        np.testing.assert_array_equal(hc[r + 1], lib.to_numpy_u64(lib.count(lib.graph_from(gr), compact)))


def test_compact_rejects_cells_and_other_k(lib, tables):
    _, compact = tables
    g = syn.chung_lu_digraph(60, 150, 2.2, None, 0.1, 5)
    dg = lib.graph_from(g)
    with pytest.raises(lib.MotifsError):
        lib.count_tuned(dg, compact, method=lib.METHOD_CELLS)
    with pytest.raises(lib.MotifsError):
        lib.table_build(5, compact=True)
    with pytest.raises(lib.MotifsError):
        compact.entries(199 << XLOW, 1)
