"""The benchmark's reference arm (the CPU oracle timed on the host): its JSON
line carries the keys the comparison needs, on rank 0 only.  The oracle's
timing and the sweep's images are replaced by stand-ins here; the arm's own
logic (steps, warm-up, line assembly) runs as written."""
import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import glcm_synth  # noqa: E402


def _args(steps=3, warmup=2):
    return argparse.Namespace(gpus=1, steps=steps, warmup=warmup, impl="reference")


def test_reference_line(monkeypatch, capsys):
    calls = []

    def fake_sample(jobs, seconds):
        calls.append(seconds)
        return 0.5 + len(calls), f"fake sample {len(calls)}"

    monkeypatch.setattr(glcm_synth, "contention_jobs", lambda side: [{"image": None}])
    monkeypatch.setattr(bench, "oracle_sample", fake_sample)
    monkeypatch.delenv("RANK", raising=False)
    assert bench.run_reference(_args()) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert len(calls) == 5  # 2 warm-up + 3 timed
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True and line["steps"] == 3 and line["warmup"] == 2
    assert line["value"] == (3.5 + 4.5 + 5.5) / 3  # the timed steps only
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"] == bench.WORKLOAD


def test_reference_other_ranks_print_nothing(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(bench, "oracle_sample", lambda *a: (_ for _ in ()).throw(AssertionError("ran")))
    assert bench.run_reference(_args()) == 0
    assert capsys.readouterr().out == ""
