"""The C ABI library builds, loads and exports the declared symbols (no GPU)."""
import ctypes as C

import numpy as np
import pytest


@pytest.fixture(scope="module")
def rs():
    from paper_1910_06416_gb300 import build
    build.build()
    import paper_1910_06416_gb300.recsplit as rs
    rs.lib()
    return rs


def test_library_exports_every_declared_function(rs):
    names = rs.header_functions()
    assert len(names) >= 13
    raw = C.CDLL(rs.LIB_PATH)
    for name in names:
        assert hasattr(raw, name), name


def test_binding_has_the_c_names(rs):
    for name in rs.header_functions():
        assert callable(getattr(rs, name)), name


def test_error_strings(rs):
    for code in (rs.OK, rs.E_INVALID, rs.E_DUPLICATE, rs.E_SEARCH_LIMIT, rs.E_NOMEM, rs.E_CUDA):
        assert rs.recsplit_strerror(code)
    assert rs.recsplit_strerror(-99) == "unknown error"


def test_invalid_arguments_rejected_before_device_work(rs):
    keys = np.arange(10, dtype=np.uint64)
    for leaf, b in [(0, 5), (25, 5), (5, 0), (5, 65536)]:
        with pytest.raises(rs.RecSplitError) as e:
            rs.recsplit_build_u64(keys, leaf, b)
        assert e.value.code == rs.E_INVALID
    with pytest.raises(rs.RecSplitError):
        rs.recsplit_deserialize(np.zeros(3, dtype=np.uint64))
    bad = np.zeros(16, dtype=np.uint64)
    bad[0] = 0x1234
    with pytest.raises(rs.RecSplitError):
        rs.recsplit_deserialize(bad)


def test_golomb_rice_table_equals_oracle(rs, orc):
    """The library derives its Golomb-Rice table independently of the oracle;
    both must agree on every node size (Eq. gr below 2^16, Sec. 7.2 above)."""
    for leaf in range(1, 25):
        hi = 65535 if leaf in (1, 5, 8, 16, 24) else 4000
        got = rs.recsplit_golomb_rice_params(leaf, hi)
        want = np.array([orc.golomb_rice(leaf, m) for m in range(hi + 1)], dtype=np.uint8)
        assert np.array_equal(got, want), leaf
    for leaf in (5, 8, 16):
        ms = [65536, 70000, 100000, 250001]
        got = rs.recsplit_golomb_rice_params(leaf, max(ms))
        assert [int(got[m]) for m in ms] == [orc.golomb_rice(leaf, m) for m in ms]


def test_golomb_rice_table_with_leaf_extra_equals_oracle(rs, orc):
    """The same for the perfect, non-minimal variant (leaf ranges m + e)."""
    for leaf, extra in [(2, 1), (5, 1), (8, 2), (8, 8), (12, 4), (16, 16), (24, 8)]:
        got = rs.recsplit_golomb_rice_params_extra(leaf, extra, 3000)
        want = np.array([orc.golomb_rice(leaf, m, extra=extra) for m in range(3001)], dtype=np.uint8)
        assert np.array_equal(got, want), (leaf, extra)
    assert np.array_equal(rs.recsplit_golomb_rice_params_extra(8, 0, 500), rs.recsplit_golomb_rice_params(8, 500))
    with pytest.raises(rs.RecSplitError):
        rs.recsplit_golomb_rice_params_extra(24, 9, 10)  # leaf + extra above 32


def test_perfect_build_arguments_rejected_before_device_work(rs):
    keys = np.arange(10, dtype=np.uint64)
    with pytest.raises(rs.RecSplitError) as e:
        rs.recsplit_build_perfect_u64(keys, 24, 5, 9)
    assert e.value.code == rs.E_INVALID


def test_profiling_modes(rs):
    for mode in (0, 1, 2, True, False):
        rs.recsplit_set_profiling(mode)
    for bad in (-1, 3):
        with pytest.raises(rs.RecSplitError):
            rs.recsplit_set_profiling(bad)
    rs.recsplit_set_profiling(0)


def test_tuning_shapes_are_validated(rs):
    t = rs.recsplit_get_tuning(8)
    assert t["leaf_warps"] in (1, 2, 4, 8)
    for bad in ({"leaf_warps": 3}, {"leaf_chunk": 0}, {"leaf_chunk": 65}, {"leaf_seeds_per_lane": 16},
                {"split_warps": [1, 16, 8]}, {"leaf_two_phase": 2}):
        tt = dict(t, **bad)
        with pytest.raises(rs.RecSplitError) as e:
            rs.recsplit_set_tuning(8, tt)
        assert e.value.code == rs.E_INVALID
    with pytest.raises(rs.RecSplitError):
        rs.recsplit_get_tuning(25)


def test_binding_rejects_strided_and_mistyped_arrays(rs):
    # checked before the library is called: the C ABI reads dense arrays of
    # fixed-size elements
    keys = np.arange(20, dtype=np.uint64)
    with pytest.raises(ValueError):
        rs.recsplit_build_u64(keys[::2], 5, 5)
    with pytest.raises(ValueError):
        rs.recsplit_build_u64(keys.astype(np.uint32), 5, 5)
    data = np.zeros(16, dtype=np.uint8)
    with pytest.raises(ValueError):
        rs.recsplit_build_bytes(data, np.array([0, 8, 16], dtype=np.int32), 5, 5)
    with pytest.raises(ValueError):
        rs.recsplit_lookup_batch([0], np.zeros(4, dtype=np.uint64), np.zeros(4, dtype=np.uint64),
                                 np.zeros(4, dtype=np.uint64))
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        rs.recsplit_build_u64(torch.arange(20, dtype=torch.int64)[::2], 5, 5)
    with pytest.raises(ValueError):
        rs.recsplit_build_u64(torch.arange(20, dtype=torch.int32), 5, 5)


def test_binding_rejects_outputs_shorter_than_the_queries(rs):
    # the library writes one result per query: a shorter output array would
    # be written past its end, so the binding raises before calling it
    keys = np.arange(8, dtype=np.uint64)
    short = np.zeros(7, dtype=np.uint64)
    data = np.zeros(64, dtype=np.uint8)
    offs = np.arange(0, 72, 8, dtype=np.uint64)  # 8 strings
    for call in (lambda: rs.recsplit_lookup_u64(0, keys, short),
                 lambda: rs.recsplit_lookup(0, keys, short),
                 lambda: rs.recsplit_lookup_u64_static(0, keys, short),
                 lambda: rs.recsplit_lookup_bytes(0, data, offs, short),
                 lambda: rs.recsplit_lookup_batch([0], np.zeros(8, dtype=np.uint32), keys, short),
                 lambda: rs.recsplit_lookup_batch([0], np.zeros(7, dtype=np.uint32), keys, np.zeros(8, np.uint64)),
                 lambda: rs.recsplit_server_submit_lookup_u64(0, 1, keys, short),
                 lambda: rs.recsplit_server_submit_lookup_bytes(0, 1, data, offs, short),
                 lambda: rs.recsplit_lookup_u64(0, keys, None)):
        with pytest.raises(ValueError):
            call()
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        rs.recsplit_lookup_u64(0, keys, torch.zeros(7, dtype=torch.int64))
