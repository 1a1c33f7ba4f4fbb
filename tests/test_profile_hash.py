"""The benchmark reports the vote kernel's DRAM traffic from the committed ncu
summary only while the kernel's code is the code that was captured: the hash
ignores // comments and blank lines, and any code change invalidates it."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_hash_ignores_comments_only():
    src = "int a = 1;  // one\n\n// a note\nint b = 2;\n"
    assert bench.code_sha256(src) == bench.code_sha256("int a = 1;\nint b = 2;  // two\n")
    assert bench.code_sha256(src) != bench.code_sha256("int a = 1;\nint b = 3;\n")


def test_committed_profile_matches_vote_source():
    assert bench.profiled_traffic("vote_contention_4096.md") is not None
