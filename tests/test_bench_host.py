"""Host logic of bench.py that needs no GPU: the DRAM-traffic record is used
only while it was captured on the current kernel sources, and it scales to
the cells of a launch."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _with_record(tmp_path, monkeypatch, rec, sha="a" * 16):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "ncu_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_sources_sha", lambda: sha)


def test_sources_hash_is_stable():
    assert bench.kernel_sources_sha() == bench.kernel_sources_sha()
    assert len(bench.kernel_sources_sha()) == 16


def test_traffic_record_used_on_matching_sources(tmp_path, monkeypatch):
    _with_record(tmp_path, monkeypatch, {"sources_sha": "a" * 16, "stage_bytes_per_cell": {"tgv256": 52.0}})
    assert bench.ncu_traffic("tgv256", 1000) == 52000.0
    assert bench.ncu_traffic("hit384", 1000) is None  # no record for that workload


def test_traffic_record_dropped_when_sources_changed(tmp_path, monkeypatch):
    _with_record(tmp_path, monkeypatch, {"sources_sha": "0" * 16, "stage_bytes_per_cell": {"tgv256": 52.0}})
    assert bench.ncu_traffic("tgv256", 1000) is None


def test_missing_traffic_record(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("tgv256", 1000) is None


def test_job_value_is_whole_job_throughput():
    # 2 ranks x 1000 cells x 10 steps in 100 ms
    assert bench.job_value(2, 1000, 10, 100.0) == 2 * 1000 * 10 / 0.1
