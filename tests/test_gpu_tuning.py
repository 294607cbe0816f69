"""Tuned launches (block size, stack depth, root-split threshold) and the
autotuner: every setting gives the automatic launch's histogram; a stack that
is too shallow is detected, never silently wrong.  GPU only."""
import numpy as np
import pytest

import oracle
import synthetic as syn
from gpu_helpers import oracle_dense

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def t5():
    import paper_1804_09741_gb300 as mt
    mt.load_library()
    return mt.table_build(5)


@pytest.mark.parametrize("scale,wpb,cap", [(0.25, 8, 0), (8.0, 32, 0), (1.0, 16, 300),
                                           (0.2, 1, 0)])
def test_tuned_launch_equals_oracle(t5, scale, wpb, cap):
    import paper_1804_09741_gb300 as mt
    g = syn.chung_lu_digraph(220, 700, 2.1, None, 0.2, 31)
    dg = mt.graph_from(g)
    h = mt.to_numpy_u64(mt.count_tuned(dg, t5, 0.0, wpb, split_scale=scale, stack_cap=cap))
    assert mt.count_stats(dg)[1] == 0
    np.testing.assert_array_equal(h, oracle_dense(oracle.count(g, 5)[0], t5.class_masks()))


def test_shallow_stack_is_reported(t5):
    import paper_1804_09741_gb300 as mt
    g = syn.workload_graph("nullmodel_k5")
    dg = mt.graph_from(g)
    mt.count_tuned(dg, t5, 0.0, 8, stack_cap=40)
    items, err, ms = mt.count_stats(dg)
    assert err != 0
    with pytest.raises(mt.MotifsError) as ei:
        out = np.empty(t5.num_classes, np.uint64)
        tun = mt.make_tuning(0.0, 8, 0.0, 40)
        import ctypes
        st = mt._lib.mt_count_tuned(dg.handle, t5.handle, out.ctypes.data, ctypes.byref(tun),
                                    None)
        mt._check(st, "mt_count_tuned")
    assert ei.value.status == mt.MT_EOVERFLOW
    # the caller's retry with a deep enough stack (automatic: (k-2) d_max + 32) is exact
    again = mt.to_numpy_u64(mt.count_tuned(dg, t5, 0.0, 8, stack_cap=0))
    assert mt.count_stats(dg)[1] == 0
    np.testing.assert_array_equal(again, mt.count_host(dg, t5))


def test_batch_with_tuning_equals_default(t5):
    import paper_1804_09741_gb300 as mt
    g = syn.chung_lu_digraph(150, 480, 2.3, None, 0.1, 8)
    dg = mt.graph_from(g)
    seeds = np.arange(1, 6, dtype=np.uint64)
    h0, z0 = mt.Batch(dg, t5, 5, 10 * g.m).run(seeds)
    h1, z1 = mt.Batch(dg, t5, 5, 10 * g.m, mt.make_tuning(0, 8, 0.5, 0)).run(seeds)
    np.testing.assert_array_equal(mt.to_numpy_u64(h0), mt.to_numpy_u64(h1))
    np.testing.assert_array_equal(z0.cpu().numpy(), z1.cpu().numpy())


def test_autotuner_picks_a_valid_launch_and_caches_it(t5, tmp_path):
    import paper_1804_09741_gb300 as mt
    from paper_1804_09741_gb300 import autotune
    g = syn.workload_graph("nullmodel_k5")
    dg = mt.graph_from(g)
    path = str(tmp_path / "tune.json")
    p = autotune.tune(dg, t5, graph=g, reps=1, cache_path=path)
    assert p.ms > 0
    again = autotune.tune(dg, t5, graph=g, reps=1, cache_path=path)
    assert again == p
    h = mt.to_numpy_u64(mt.count_tuned(dg, t5, 0.0, p.warps_per_block, split_scale=p.split_scale,
                                       stack_cap=p.stack_cap))
    np.testing.assert_array_equal(h, mt.to_numpy_u64(mt.count(dg, t5)))


def test_batch_autotuner_keeps_histograms(t5, tmp_path):
    import paper_1804_09741_gb300 as mt
    from paper_1804_09741_gb300 import autotune
    g = syn.chung_lu_digraph(300, 1000, 2.2, None, 0.1, 12)
    dg = mt.graph_from(g)
    path = str(tmp_path / "b.json")
    p = autotune.tune_batch(dg, t5, g, 10 * g.m, probe_nulls=4, cache_path=path)
    assert p.warps_per_block in (16, 32) and p.ms > 0
    assert autotune.tune_batch(dg, t5, g, 10 * g.m, probe_nulls=4, cache_path=path) == p
    seeds = np.arange(1, 5, dtype=np.uint64)
    h0, _ = mt.Batch(dg, t5, 4, 10 * g.m).run(seeds)
    h1, _ = mt.Batch(dg, t5, 4, 10 * g.m, p.tuning()).run(seeds)
    np.testing.assert_array_equal(mt.to_numpy_u64(h0), mt.to_numpy_u64(h1))


def test_probe_rates_are_measured():
    import paper_1804_09741_gb300 as mt
    g, a = mt.probe_rates(1 << 20, 1 << 14)
    assert 1e9 < g < 1e14 and 1e8 < a < 1e14
    with pytest.raises(mt.MotifsError):
        mt.probe_rates(1000, 1 << 14)  # not a power of two


def test_expired_idle_wait_reports_timeout(t5):
    """Fault injection from the host: with an idle-wait limit of a few
    nanoseconds, warps that run out of work before their block-mates give up
    and the count reports MT_ETIMEOUT (no GPU fault, trap or hang); with the
    limit restored the same count is exact again."""
    import paper_1804_09741_gb300 as mt
    g = syn.workload_graph("nullmodel_k5")
    dg = mt.graph_from(g)
    want = mt.count_host(dg, t5)
    try:
        mt.set_wait_limit(5)
        with pytest.raises(mt.MotifsError) as err:
            mt.count_host(dg, t5)
        assert err.value.status == mt.MT_ETIMEOUT
    finally:
        mt.set_wait_limit(0)
    np.testing.assert_array_equal(mt.count_host(dg, t5), want)
