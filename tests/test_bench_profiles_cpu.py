"""bench.py reads DRAM traffic and utilisation counters from the ncu summaries
under profiles/ only while the kernel source they were captured from is
unchanged (its hash is recorded in the summary)."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

SUMMARY = """# test kernel

- source_sha256_16: `{sha}`
- dram_bytes_per_launch: `1234`
- dram_bytes_all_launches: `5678`

| metric | unit | launch 1 |
|---|---|---|
| smsp__issue_active.avg.pct_of_peak_sustained_active | % | 75.5 |
| gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed | % | 1.25 |
"""


def make_tree(tmp_path, source_text, recorded_sha):
    csrc = tmp_path / "paper_1910_06416_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text(source_text)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k_test.md").write_text(SUMMARY.format(sha=recorded_sha))


def test_counters_are_read_while_the_source_is_unchanged(tmp_path, monkeypatch):
    src = "__global__ void k() {}\n"
    make_tree(tmp_path, src, hashlib.sha256(src.encode()).hexdigest()[:16])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profiles("k_test", "k.cu") == 1234.0
    assert bench.traffic_from_profiles("k_test", "k.cu", key="dram_bytes_all_launches") == 5678.0
    assert bench.counters_from_profiles("k_test", "k.cu") == {"issue_active_pct": 75.5, "dram_throughput_pct": 1.25}


def test_counters_are_dropped_once_the_source_changes(tmp_path, monkeypatch):
    make_tree(tmp_path, "__global__ void k() { /* changed */ }\n", "0123456789abcdef")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profiles("k_test", "k.cu") is None
    assert bench.counters_from_profiles("k_test", "k.cu") is None
    assert bench.traffic_from_profiles("missing", "k.cu") is None
