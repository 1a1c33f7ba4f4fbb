"""The serving arena's allocator (host C++), compiled with g++ and checked
against a byte-map model on random alloc/free sequences."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def arena_bin(tmp_path_factory):
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("no g++")
    out = str(tmp_path_factory.mktemp("arena") / "arena_check")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "paper_1710_06189_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "arena_check.cpp"), "-o", out], check=True)
    return out


@pytest.mark.parametrize("seed", [1, 2, 3, 20171018])
def test_first_fit_matches_model(arena_bin, seed):
    r = subprocess.run([arena_bin, str(seed)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("OK")
