"""bench.py reads DRAM traffic and utilisation counters from the ncu summaries
under profiles/ only while the kernel source they were captured from, and the
shared headers it includes, are unchanged (their hash is recorded in the
summary)."""
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


HEADER = "__device__ int f() { return 1; }\n"


def make_tree(tmp_path, source_text, recorded_sha):
    csrc = tmp_path / "paper_1910_06416_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text(source_text)
    (csrc / "device.cuh").write_text(HEADER)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k_test.md").write_text(SUMMARY.format(sha=recorded_sha))
    return csrc


def sha_of(*texts):
    h = hashlib.sha256()
    for t in texts:
        h.update(t.encode())
    return h.hexdigest()[:16]


def test_counters_are_read_while_the_source_is_unchanged(tmp_path, monkeypatch):
    src = "__global__ void k() {}\n"
    make_tree(tmp_path, src, sha_of(src, HEADER))
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


def test_counters_are_dropped_once_a_shared_header_changes(tmp_path, monkeypatch):
    src = "__global__ void k() {}\n"
    csrc = make_tree(tmp_path, src, sha_of(src, HEADER))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profiles("k_test", "k.cu") == 1234.0
    (csrc / "device.cuh").write_text(HEADER + "// changed\n")
    assert bench.traffic_from_profiles("k_test", "k.cu") is None
