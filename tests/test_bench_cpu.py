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
