"""The tuning cache on the host: entries keyed by GPU, leaf size and bucket
size round-trip through the JSON file and are installed with
recsplit_set_tuning (no device work)."""
import json

import pytest

from paper_1910_06416_gb300 import tuning_cache as tc


@pytest.fixture(scope="module")
def rs():
    from paper_1910_06416_gb300 import build
    build.build()
    import paper_1910_06416_gb300.recsplit as rs
    rs.lib()
    return rs


def test_cache_round_trip_and_install(rs, tmp_path):
    path = str(tmp_path / "t.json")
    shape = {"leaf_warps": 2, "leaf_chunk": 16, "leaf_seeds_per_lane": 2, "split_warps": [1, 2, 4],
             "leaf_two_phase": 1}
    assert tc.install("GB300", 11, 100, path) is None  # nothing cached yet
    tc.save({tc.cache_key("GB300", 11, 100): shape}, path)
    assert tc.load(path) == {"GB300|l=11|b=100": shape}
    before = rs.recsplit_get_tuning(11)
    try:
        assert tc.install("GB300", 11, 100, path) == shape
        assert rs.recsplit_get_tuning(11) == shape
        assert tc.install("other GPU", 11, 100, path) is None  # keyed by device
        assert tc.install("GB300", 11, 5, path) is None  # and by bucket size
    finally:
        rs.recsplit_set_tuning(11, before)


def test_invalid_or_damaged_entries_are_ignored(rs, tmp_path):
    path = str(tmp_path / "t.json")
    bad = {"leaf_warps": 3, "leaf_chunk": 4, "leaf_seeds_per_lane": 1, "split_warps": [1, 1, 8],
           "leaf_two_phase": 0}  # 3 warps: not a power of two
    tc.save({tc.cache_key("GB300", 9, 100): bad}, path)
    before = rs.recsplit_get_tuning(9)
    assert tc.install("GB300", 9, 100, path) is None
    assert rs.recsplit_get_tuning(9) == before
    with open(path, "w") as f:
        f.write("{not json")
    assert tc.load(path) == {}
    with open(path, "w") as f:
        json.dump([1, 2], f)
    assert tc.load(path) == {}
