"""Launch shapes (and the autotuner that picks them) change speed only: the
structures stay identical to the oracle's under any valid shape."""
import numpy as np
import pytest

from paper_1910_06416_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1910_06416_gb300 import build
    build.build()
    import paper_1910_06416_gb300.recsplit as rs
    rs.lib()
    return rs


SHAPES = [
    {"leaf_warps": 1, "leaf_chunk": 1, "leaf_seeds_per_lane": 1, "split_warps": [1, 1, 1], "leaf_two_phase": 0},
    {"leaf_warps": 8, "leaf_chunk": 64, "leaf_seeds_per_lane": 8, "split_warps": [8, 8, 8], "leaf_two_phase": 1},
    {"leaf_warps": 2, "leaf_chunk": 16, "leaf_seeds_per_lane": 2, "split_warps": [2, 4, 2], "leaf_two_phase": 1},
    {"leaf_warps": 4, "leaf_chunk": 4, "leaf_seeds_per_lane": 1, "split_warps": [1, 2, 8], "leaf_two_phase": 1},
]


@pytest.mark.parametrize("leaf,b,n", [(8, 100, 40000), (5, 5, 20000), (12, 200, 6000), (16, 2000, 5000)])
def test_structures_identical_under_every_shape(rs, orc, leaf, b, n):
    keys = inputs.u64_keys(n, 100 + leaf)
    ref = orc.build_u64(keys, leaf, b, threads=8)
    saved = rs.recsplit_get_tuning(leaf)
    try:
        for shape in SHAPES:
            rs.recsplit_set_tuning(leaf, shape)
            got = rs.Structure.build_u64(torch.from_numpy(keys.view(np.int64)).cuda(), leaf, b).serialize()
            assert np.array_equal(got, ref), shape
    finally:
        rs.recsplit_set_tuning(leaf, saved)


def test_autotuner_installs_valid_shapes(rs, orc):
    t = rs.recsplit_autotune(8, 100, 1 << 18)
    assert rs.recsplit_get_tuning(8) == t
    assert t["leaf_warps"] in (1, 2, 4, 8) and t["leaf_seeds_per_lane"] in (1, 2, 4, 8)
    keys = inputs.u64_keys(30000, 7)
    got = rs.Structure.build_u64(keys, 8, 100).serialize()
    assert np.array_equal(got, orc.build_u64(keys, 8, 100))
