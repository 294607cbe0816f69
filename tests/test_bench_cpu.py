"""Host-side helpers of bench.py (no GPU): the comment-insensitive kernel
source hash that keys the committed traffic evidence."""
import bench


def test_strip_comments_ignores_comments_and_whitespace():
    a = "int x = 1;  // one\n/* block\n comment */ int y = 2;\n"
    b = "int x = 1;\n\n   int y = 2; // two\n"
    assert bench._strip_comments(a) == bench._strip_comments(b) == "int x = 1; int y = 2;"


def test_strip_comments_keeps_code_changes_and_literals():
    assert bench._strip_comments("int x = 1;") != bench._strip_comments("int x = 2;")
    src = 'const char* s = "a // b /* c */";  char q = \'"\'; // gone'
    out = bench._strip_comments(src)
    assert '"a // b /* c */"' in out and "'\"'" in out and "gone" not in out


def test_kernel_source_hash_is_stable():
    h = bench._kernel_source_hash()
    assert len(h) == 16 and h == bench._kernel_source_hash()


def test_captured_counters_apply_only_to_the_current_source(tmp_path, monkeypatch):
    import json
    src = bench._kernel_source_hash()
    p = tmp_path / "c.json"
    p.write_text(json.dumps({"captures": [
        {"kind": "traffic", "method": "enumerate", "workload": "w", "nulls": 4, "source": src,
         "dram_bytes": 123},
        {"kind": "traffic", "method": "enumerate", "workload": "w", "nulls": 8,
         "source": "0000000000000000", "dram_bytes": 456}]}))
    monkeypatch.setattr(bench, "COUNTERS_JSON", str(p))
    assert bench._captured_traffic("enumerate", "w", 4) == 123
    assert bench._captured_traffic("enumerate", "w", 8) is None  # another kernel source
    assert bench._captured_traffic("cells", "w", 4) is None


def test_committed_counters_file_is_valid_json():
    import json
    with open(bench.COUNTERS_JSON) as f:
        d = json.load(f)
    for e in d["captures"]:
        assert {"kind", "method", "workload", "source"} <= set(e)
