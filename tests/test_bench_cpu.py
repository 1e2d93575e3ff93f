"""Host logic of bench.py that needs no GPU: the comment-insensitive hash
that ties the headline's DRAM traffic to the kernels it was measured on, and
the lookup of that traffic in the committed ncu summary."""
import os

import bench


def test_code_only_drops_comments_and_blank_lines():
    src = "int a = 1;  // note\n\n/* block\n   comment */ int b = 2;\n    // only a comment\nint c;\n"
    assert bench._code_only(src) == "int a = 1;\n int b = 2;\nint c;"


def test_replay_hash_ignores_comment_edits_only():
    path = os.path.join(bench.ROOT, "paper_1907_07875_gb300", "csrc", bench.REPLAY_SOURCES[2])
    text = open(path).read()
    assert bench._code_only(text) == bench._code_only("// a new comment\n" + text.replace("\n", "  // x\n", 3))
    assert bench._code_only(text) != bench._code_only(text.replace("{", "{ ;", 1))


def test_replay_traffic_lookup():
    t = bench._replay_traffic()
    assert t is None or (isinstance(t, int) and t > 0)
