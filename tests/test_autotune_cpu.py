"""Autotuner host logic without a GPU: profile keys and the JSON cache."""
import synthetic as syn
from paper_1804_09741_gb300 import autotune


def test_profile_key_groups_a_family():
    g = syn.chung_lu_digraph(1500, 6000, 2.2, None, 0.1, 0)
    h = syn.chung_lu_digraph(1500, 6000, 2.2, None, 0.1, 1)
    assert autotune.degree_profile(g, 5) == autotune.degree_profile(h, 5)
    assert autotune.degree_profile(g, 5) != autotune.degree_profile(g, 6)
    u = syn.uniform_digraph(1500, 6000, 0)
    assert autotune.degree_profile(u, 5) != autotune.degree_profile(g, 5)


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "c" / "t.json")
    assert autotune.load_cache(path) == {}
    autotune.save_cache({"k5-x": {"warps_per_block": 16, "split_scale": 0.5, "stack_cap": 0,
                                  "ms": 1.0}}, path)
    c = autotune.load_cache(path)
    assert autotune.TuneParams(**c["k5-x"]).warps_per_block == 16


def test_candidates_cover_block_split_and_stack():
    cs = list(autotune.candidates(261, 5))
    assert {c.warps_per_block for c in cs} == {8, 16, 32}
    assert {c.split_scale for c in cs} >= {0.25, 1.0, 8.0}
    assert any(c.stack_cap > 0 for c in cs) and any(c.stack_cap == 0 for c in cs)
