"""The benchmark reports the vote kernels' DRAM traffic from the committed ncu
summary only while their code is the code that was captured: the hash covers
every vote source, ignores // comments and blank lines, and any code change
invalidates it."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_hash_ignores_comments_only():
    src = "int a = 1;  // one\n\n// a note\nint b = 2;\n"
    assert bench.code_sha256(src) == bench.code_sha256("int a = 1;\nint b = 2;  // two\n")
    assert bench.code_sha256(src) != bench.code_sha256("int a = 1;\nint b = 3;\n")


def test_traffic_reported_only_for_the_captured_code(tmp_path, monkeypatch):
    """profiled_traffic() gives the summary's figure when its hash is the
    current source's, and None (traffic unknown) once the code has changed."""
    good = bench.vote_code_sha256()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "cur.md").write_text(f"traffic_bytes_per_step: 1234\nvote_code_sha256: {good}\n")
    (prof / "old.md").write_text("traffic_bytes_per_step: 1234\nvote_code_sha256: " + "0" * 64 + "\n")
    real_join = os.path.join

    def join(*parts):
        if len(parts) >= 2 and parts[0] == bench.ROOT and parts[1] == "profiles":
            return real_join(str(prof), *parts[2:])
        return real_join(*parts)

    monkeypatch.setattr(bench.os.path, "join", join)
    assert bench.profiled_traffic("cur.md") == 1234.0
    assert bench.profiled_traffic("old.md") is None
    assert bench.profiled_traffic("missing.md") is None


def test_vote_hash_covers_every_vote_source():
    csrc = os.path.join(ROOT, "paper_1710_06189_gb300", "csrc")
    for f in bench.VOTE_SOURCES:
        assert os.path.exists(os.path.join(csrc, f)), f
    assert set(bench.VOTE_SOURCES) >= {"vote.cu", "vote_fast.cuh"}
