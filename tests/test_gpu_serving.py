"""The continuous-batching server: every result equals the same graph counted
alone (bit-exact), requests arriving mid-flight overtake a long one, memory
budget and slots bound admission, bad requests fail alone.  GPU only."""
import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tables():
    import paper_1804_09741_gb300 as mt
    mt.load_library()
    return {k: mt.table_build(k) for k in (3, 4, 5, 6)}


def alone(mt, t, g):
    return mt.count_host(mt.graph_from(g), t)


@pytest.mark.parametrize("method", [0, 1])
def test_mixed_stream_equals_alone(tables, method):
    import paper_1804_09741_gb300 as mt
    from paper_1804_09741_gb300.server import Server, poisson_arrivals, run_stream
    reqs = []
    rng = np.random.default_rng(3)
    for i in range(24):
        k = [3, 4, 5, 6][i % 4]
        n = int(rng.integers(30, 900 if k < 6 else 300))
        g = syn.chung_lu_digraph(n, int(n * rng.uniform(2, 4)), 2.3, 30, 0.2, 1000 + i)
        reqs.append((k, g))
    reqs += [(4, syn.empty_graph(7)), (5, syn.empty_graph(1)), (6, syn.complete_digraph(5)),
             (3, syn.complete_digraph(9))]
    srv = Server(tables, memory_budget=2 << 30, max_slots=8, round_cost=2e6, method=method)
    out, lat, wall = run_stream(srv, reqs, poisson_arrivals(len(reqs), 400.0, 1))
    for (k, g), (st, hist, status) in zip(reqs, out):
        assert st == 2, status
        np.testing.assert_array_equal(hist, alone(mt, tables[k], g))
    assert np.all(lat > 0)
    assert srv.used_bytes() == 0
    srv.free()


def test_late_small_requests_overtake_a_long_one(tables):
    import paper_1804_09741_gb300 as mt
    from paper_1804_09741_gb300.server import Server
    big = syn.workload_graph("nullmodel_k5")
    srv = Server(tables, memory_budget=4 << 30, max_slots=16, round_cost=2e7)
    bid = srv.submit(5, big)
    for _ in range(3):
        srv.step()
    small = [syn.chung_lu_digraph(200, 600, 2.3, 20, 0.1, 50 + i) for i in range(4)]
    sids = [srv.submit(4, g) for g in small]
    done_small, big_done_at, step = {}, None, 0
    results = {}
    while big_done_at is None or len(done_small) < 4:
        srv.step()
        step += 1
        for sid, g in zip(sids, small):
            if sid not in done_small:
                st, h, ms, _ = srv.result(sid, 4)
                if st == 2:
                    done_small[sid] = step
                    results[sid] = h
        if big_done_at is None:
            st, h, ms, _ = srv.result(bid, 5)
            if st == 2:
                big_done_at = step
                big_hist = h
        assert step < 100000
    assert max(done_small.values()) < big_done_at  # admitted mid-flight, finished first
    np.testing.assert_array_equal(big_hist, alone(mt, tables[5], big))
    for sid, g in zip(sids, small):
        np.testing.assert_array_equal(results[sid], alone(mt, tables[4], g))
    srv.free()


def test_budget_and_slots_bound_admission(tables):
    """The budget covers the requests' memory and their k's round scratch
    (planner, work queue, graph descriptors): with room for two requests plus
    the scratch of a two-request round, at most two run at once, the charge
    never exceeds the budget, and it returns to zero when all are done."""
    import paper_1804_09741_gb300 as mt
    from paper_1804_09741_gb300.server import Server, run_stream
    graphs = [syn.chung_lu_digraph(800, 3000, 2.4, 40, 0.1, 70 + i) for i in range(6)]
    # request bytes as the server charges them: graph arrays, histogram, planner share
    per = 4 * (3 * 801 + 5 * 3000) + 64 * 3800 + 13 * 8 + 4096
    probe = Server(tables, memory_budget=1 << 34, max_slots=2, round_cost=1e6)
    for g in graphs[:2]:
        probe.submit(3, g)
    probe.step()
    two = probe.used_bytes()
    assert two > 2 * per  # the round scratch is charged beside the requests
    probe.free()
    budget = two + 1000
    srv = Server(tables, memory_budget=budget, max_slots=3, round_cost=1e6)
    ids = [srv.submit(3, g) for g in graphs]
    seen_pending, max_active = False, 0
    remaining = set(ids)
    res = {}
    while remaining:
        c, a, p = srv.step()
        max_active = max(max_active, a)
        seen_pending |= p > 0
        assert srv.used_bytes() <= budget
        for rid in list(remaining):
            st, h, ms, _ = srv.result(rid, 3)
            if st == 2:
                res[rid] = h
                remaining.discard(rid)
    assert seen_pending and max_active <= 2
    assert srv.used_bytes() == 0  # scratch of an idle k is released
    for rid, g in zip(ids, graphs):
        np.testing.assert_array_equal(res[rid], alone(mt, tables[3], g))
    # a request that can never fit the budget fails on its own
    bid = srv.submit(6, syn.workload_graph("nullmodel_k6"))
    for _ in range(3):
        srv.step()
    st, h, ms, status = srv.result(bid, 6)
    assert st == 3 and status == mt.MT_EBUSY
    srv.free()


def test_launch_errors_fail_their_requests(tables):
    """Fault injection from the host (no GPU fault, trap or hang): with an
    idle-wait limit of a few nanoseconds the rounds' launches report an expired
    wait, and every request that had a chunk in such a launch fails with
    MT_ETIMEOUT instead of returning a histogram that may be incomplete; with
    the limit restored the same requests are served exactly."""
    import paper_1804_09741_gb300 as mt
    from paper_1804_09741_gb300.server import Server, run_stream
    reqs = [(5, syn.workload_graph("nullmodel_k5")), (4, syn.workload_graph("chunglu_k4"))]
    srv = Server(tables, memory_budget=4 << 30, max_slots=8, round_cost=1e12)
    try:
        mt.set_wait_limit(5)
        out, lat, wall = run_stream(srv, reqs)
    finally:
        mt.set_wait_limit(0)
    assert out[0][0] == 3 and out[0][1] is None and out[0][2] == mt.MT_ETIMEOUT
    assert srv.used_bytes() == 0
    out, lat, wall = run_stream(srv, reqs)
    for (k, g), (st, hist, status) in zip(reqs, out):
        assert st == 2, status
        np.testing.assert_array_equal(hist, alone(mt, tables[k], g))
    srv.free()


def test_bad_request_fails_alone(tables):
    import paper_1804_09741_gb300 as mt
    from paper_1804_09741_gb300.server import Server, run_stream
    dup = syn.Graph(3, np.array([0, 2, 2, 2], np.int32), np.array([1, 1], np.int32))
    good = syn.chung_lu_digraph(300, 900, 2.3, 30, 0.1, 5)
    srv = Server(tables, round_cost=1e6)
    out, lat, wall = run_stream(srv, [(4, good), (4, dup), (4, good)])
    assert out[1][0] == 3 and out[1][2] == mt.MT_EINVAL
    for i in (0, 2):
        assert out[i][0] == 2
        np.testing.assert_array_equal(out[i][1], alone(mt, tables[4], good))
    with pytest.raises(mt.MotifsError):
        srv.submit(4, syn.Graph(2, np.array([0, 1, 1], np.int32), np.array([0], np.int32)))
    srv.free()


def test_unsupported_table_method_pair_fails_alone(tables):
    """The cell method cannot use a compact k = 6 table: the server fails those
    requests alone (status MT_EUNSUPPORTED, no partial result) and serves the
    others in the same rounds."""
    import paper_1804_09741_gb300 as mt
    from paper_1804_09741_gb300.server import Server, run_stream
    compact6 = mt.table_build(6, compact=True)
    srv = Server({5: tables[5], 6: compact6}, memory_budget=2 << 30, max_slots=8,
                 round_cost=2e6, method=mt.METHOD_CELLS)
    g5 = syn.chung_lu_digraph(400, 1200, 2.3, 30, 0.2, 7)
    g6 = syn.chung_lu_digraph(120, 360, 2.3, 20, 0.2, 8)
    reqs = [(6, g6), (5, g5), (6, g6)]
    out, lat, wall = run_stream(srv, reqs)
    assert out[0][0] == 3 and out[0][2] == mt.MT_EUNSUPPORTED and out[0][1] is None
    assert out[2][0] == 3 and out[2][2] == mt.MT_EUNSUPPORTED
    assert out[1][0] == 2
    np.testing.assert_array_equal(out[1][1], alone(mt, tables[5], g5))
    assert srv.used_bytes() == 0
    srv.free()
    compact6.free()


def test_compact_k6_table_in_the_server(tables):
    """The per-subgraph method serves k = 6 requests from the compact table;
    results equal the full table's one-graph counts."""
    import paper_1804_09741_gb300 as mt
    from paper_1804_09741_gb300.server import Server, poisson_arrivals, run_stream
    compact6 = mt.table_build(6, compact=True)
    srv = Server({5: tables[5], 6: compact6}, memory_budget=2 << 30, max_slots=8,
                 round_cost=2e6)
    reqs = [(6, syn.chung_lu_digraph(n, 3 * n, 2.3, 20, 0.2, 40 + n)) for n in (60, 150, 240)]
    reqs.append((5, syn.chung_lu_digraph(300, 900, 2.3, 30, 0.2, 9)))
    out, lat, wall = run_stream(srv, reqs, poisson_arrivals(len(reqs), 300.0, 2))
    for (k, g), (st, hist, status) in zip(reqs, out):
        assert st == 2, status
        np.testing.assert_array_equal(hist, alone(mt, tables[k], g))
    srv.free()
    compact6.free()
