"""Host-side helpers of the benchmark: the algorithmic-bytes model, the
percentile, the comment-insensitive kernel digest and the profile lookup."""
import os
import types

import bench


def test_algorithmic_bytes_model():
    ls = types.SimpleNamespace(expanded=4, e_scan=1000, touched=300, walk_scan=20, interior=2)
    # 2 offsets per expanded vertex, 4 B per scanned entry, 16 B per reached
    # vertex, 4 B per walk scan, 4 B per counted interior vertex
    assert bench.algorithmic_bytes(ls, 4) == 2 * 4 * 4 + 4 * 1000 + 16 * 300 + 4 * 20 + 4 * 2
    assert bench.algorithmic_bytes(ls, 8) - bench.algorithmic_bytes(ls, 4) == 2 * 4 * 4


def test_percentile_interpolates():
    xs = [5.0, 1.0, 3.0, 2.0, 4.0]
    assert bench.percentile(xs, 0) == 1.0
    assert bench.percentile(xs, 50) == 3.0
    assert bench.percentile(xs, 100) == 5.0
    assert bench.percentile([1.0, 2.0], 50) == 1.5
    assert bench.percentile([], 50) is None


def test_code_digest_ignores_comments_only():
    a = "int f(int x) {\n  return x + 1;  // one\n}\n/* block\n comment */\n"
    b = "// header\nint f(int x) {\n\n  return x + 1;\n}\n"
    c = "int f(int x) {\n  return x + 2;\n}\n"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)


def test_profile_traffic_is_used_only_for_the_current_kernel():
    digest = bench.kernel_digest()
    assert len(digest) == 16
    path = os.path.join(bench.ROOT, "profiles", "batch_kernel_rmat20.md")
    text = open(path).read()
    if f"kernel_digest: {digest}" in text:
        assert bench.profiled_traffic("rmat20", "batch_kernel") > 0
    else:
        assert bench.profiled_traffic("rmat20", "batch_kernel") is None
    assert bench.profiled_traffic("no_such_workload", "batch_kernel") is None
