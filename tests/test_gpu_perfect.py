"""Perfect, non-minimal variant on the GPU against the oracle, through the
C ABI: byte-identical structures, identical lookups, and the lookups of the
keys distinct values in [0, range_size)."""
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


def dev_u64(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def host_u64(t):
    return t.cpu().numpy().view(np.uint64)


CASES = [(5, 5, 1, 50000, 0), (8, 100, 2, 100000, 1), (8, 100, 8, 60000, 2), (12, 9, 4, 20000, 3),
         (16, 40, 6, 3000, 4), (3, 1000, 2, 20000, 5), (2, 7, 1, 5000, 6), (24, 30, 8, 1500, 7),
         (8, 100, 3, 1, 8), (8, 100, 3, 0, 9), (10, 2000, 5, 30000, 10)]


@pytest.mark.parametrize("leaf,b,extra,n,seed", CASES)
def test_perfect_u64_matches_oracle(rs, orc, leaf, b, extra, n, seed):
    keys = inputs.u64_keys(n, 60 + seed)
    ref = orc.build_u64(keys, leaf, b, threads=8, extra=extra)
    s = rs.Structure.build_perfect_u64(dev_u64(keys), leaf, b, extra)
    blob = s.serialize()
    assert blob.shape == ref.shape and np.array_equal(blob, ref)
    st = s.stats()
    assert st["leaf_extra"] == extra and st["leaf_size"] == leaf
    if n == 0:
        assert st["range_size"] == 0
        return
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    s.lookup_u64(dev_u64(keys), out)
    got = host_u64(out)
    assert np.array_equal(got, orc.lookup_u64(ref, keys))
    assert np.unique(got).shape[0] == n and int(got.max()) < st["range_size"]
    # the range is the oracle's: sum of the bucket ranges
    hi, _ = orc.fingerprint_u64(keys)
    nb = -(-n // b)
    sizes = np.bincount([orc.bucket(int(x), nb) for x in hi], minlength=nb)
    assert st["range_size"] == sum(orc.node_range(leaf, extra, int(m)) for m in sizes)
    # non-member keys: the same deterministic values as the oracle's
    others = inputs.u64_keys(n + 2000, 90 + seed)[n:]
    o2 = torch.empty(others.shape[0], dtype=torch.int64, device="cuda")
    s.lookup_u64(dev_u64(others), o2)
    assert np.array_equal(host_u64(o2), orc.lookup_u64(ref, others))


def test_perfect_bytes_and_host_buffers(rs, orc):
    bk = inputs.byte_keys(40000, 70)
    ref = orc.build_bytes(bk.data, bk.offsets, 8, 100, threads=8, extra=2)
    s = rs.Structure.build_perfect_bytes(bk.data, bk.offsets, 8, 100, 2)  # host buffers
    assert np.array_equal(s.serialize(), ref)
    out = np.zeros(40000, dtype=np.uint64)
    s.lookup_bytes(bk.data, bk.offsets, out)
    assert np.array_equal(out, orc.lookup_bytes(ref, bk.data, bk.offsets))


def test_zero_extra_is_the_minimal_structure(rs):
    keys = dev_u64(inputs.u64_keys(30000, 71))
    a = rs.Structure.build_perfect_u64(keys, 8, 100, 0).serialize()
    b = rs.Structure.build_u64(keys, 8, 100).serialize()
    assert np.array_equal(a, b)


def test_round_trip_batch_lookup_and_allocation_free_lookup(rs, orc):
    keys = inputs.u64_keys(50000, 72)
    s = rs.Structure.build_perfect_u64(dev_u64(keys), 8, 100, 3)
    blob = s.serialize()
    s2 = rs.Structure.deserialize(blob)
    assert s2.stats()["range_size"] == s.stats()["range_size"]
    want = orc.lookup_u64(blob, keys)
    out = torch.empty(keys.shape[0], dtype=torch.int64, device="cuda")
    s2.lookup_u64(dev_u64(keys), out)
    assert np.array_equal(host_u64(out), want)
    # batched lookups mixing a minimal and a perfect structure, small and
    # large batches (per-query selects and the decoded bucket table)
    mk = inputs.u64_keys(20000, 73)
    m = rs.Structure.build_u64(dev_u64(mk), 5, 5)
    mwant = orc.lookup_u64(m.serialize(), mk)
    for q in (500, 400000):
        rng = np.random.default_rng(q)
        ids = rng.integers(0, 2, q).astype(np.uint32)
        pick = np.where(ids == 0, rng.integers(0, keys.shape[0], q), rng.integers(0, mk.shape[0], q))
        qk = np.where(ids == 0, keys[pick % keys.shape[0]], mk[pick % mk.shape[0]]).astype(np.uint64)
        o = np.zeros(q, dtype=np.uint64)
        rs.recsplit_lookup_batch([s.handle, m.handle], ids, qk, o)
        exp = np.where(ids == 0, want[pick % keys.shape[0]], mwant[pick % mk.shape[0]])
        assert np.array_equal(o, exp), q
    # the allocation-free lookup reads the same structure
    o3 = np.zeros(10000, dtype=np.uint64)
    rs.recsplit_lookup_u64_static(s.handle, keys[:10000], o3)
    assert np.array_equal(o3, want[:10000])


def test_perfect_full_size_leaf8_bucket100(rs, orc):
    """10^6 keys, l = 8, b = 100, leaf range extra 2: byte-identical to the
    oracle and an injection into [0, range_size)."""
    n = 1_000_000
    keys = inputs.u64_keys(n, 74)
    s = rs.Structure.build_perfect_u64(dev_u64(keys), 8, 100, 2)
    ref = orc.build_u64(keys, 8, 100, threads=32, extra=2)
    assert np.array_equal(s.serialize(), ref)
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    s.lookup_u64(dev_u64(keys), out)
    r = s.stats()["range_size"]
    assert torch.unique(out).numel() == n and int(out.max()) < r
    sample = np.random.default_rng(5).integers(0, n, 20000)
    assert np.array_equal(host_u64(out)[sample], orc.lookup_u64(ref, keys[sample]))


def test_batched_build_mixes_minimal_and_perfect_sets(rs, orc):
    plan = [(20000, 8, 100, 0), (15000, 8, 100, 2), (30000, 5, 5, 1), (8000, 12, 9, 4), (5000, 8, 100, 0),
            (1, 8, 100, 3), (0, 5, 5, 2)]
    keys = [inputs.u64_keys(n, 80 + i) for i, (n, _, _, _) in enumerate(plan)]
    sets = [(dev_u64(k), l, b, {"leaf_extra": e}) for k, (n, l, b, e) in zip(keys, plan)]
    hs = rs.recsplit_build_batch(sets)
    try:
        for h, k, (n, l, b, e) in zip(hs, keys, plan):
            assert np.array_equal(rs.recsplit_serialize(h), orc.build_u64(k, l, b, threads=4, extra=e)), (n, l, b, e)
            assert rs.recsplit_stats(h)["leaf_extra"] == e
    finally:
        for h in hs:
            rs.recsplit_free(h)
