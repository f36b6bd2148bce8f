"""CUDA path vs the oracle, through the C ABI.

Every integer of the structure must be identical (byte-identical serialized
form) and every lookup must return the oracle's value.  At full sizes where
the oracle cannot build everything, sampled buckets are rebuilt by the oracle
from its own grouping and compared with the GPU structure decoded by the
oracle's own reader, and the lookups of all keys must form a permutation.
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest

from paper_1910_06416_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THREADS = max(1, min(32, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1910_06416_gb300 import build
    build.build()
    import paper_1910_06416_gb300.recsplit as rs
    rs.lib()
    return rs


def dev_u64(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def host_u64(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def gpu_build_u64(rs, keys, leaf, b):
    return rs.Structure.build_u64(dev_u64(keys), leaf, b)


def gpu_lookup_u64(s, keys):
    out = torch.empty(keys.shape[0], dtype=torch.int64, device="cuda")
    s.lookup_u64(dev_u64(keys), out)
    torch.cuda.synchronize()
    return host_u64(out)


def assert_same_blob(gpu, ref):
    assert gpu.shape == ref.shape, (gpu.shape, ref.shape)
    if not np.array_equal(gpu, ref):
        bad = np.nonzero(gpu != ref)[0]
        raise AssertionError(f"{bad.size} words differ, first at {bad[:8].tolist()}")


# ---------------------------------------------------------------- small cases
CASES = [(5, 5, 100000, 0), (8, 100, 30000, 3), (1, 1, 500, 4), (1, 7, 777, 5), (2, 3, 1000, 6),
         (12, 9, 3000, 7), (3, 1000, 5000, 8), (24, 1, 50, 9), (16, 40, 120, 10), (8, 100, 1, 11),
         (8, 100, 2, 12), (8, 100, 3, 13), (5, 5, 0, 14), (7, 65535, 2000, 15), (4, 16, 4097, 16),
         (10, 50, 12345, 17), (6, 3000, 9000, 18), (20, 20, 200, 19)]


@pytest.mark.parametrize("leaf,b,n,seed", CASES)
def test_u64_structure_and_lookups_match_oracle(rs, orc, leaf, b, n, seed):
    keys = inputs.u64_keys(n, seed)
    ref = orc.build_u64(keys, leaf, b)
    s = gpu_build_u64(rs, keys, leaf, b)
    assert_same_blob(s.serialize(), ref)
    if n:
        got = gpu_lookup_u64(s, keys)
        assert np.array_equal(got, orc.lookup_u64(ref, keys))
        assert np.array_equal(np.sort(got), np.arange(n, dtype=np.uint64))
    others = inputs.splitmix64(seed + 1000, 3000)
    assert np.array_equal(gpu_lookup_u64(s, others), orc.lookup_u64(ref, others))
    st = s.stats()
    assert st["n"] == n and st["num_codes"] == orc.header(ref)["codes"]


def random_configs(count=40, seed=77):
    # leaf sizes 1..12, bucket sizes log-uniform in [1, 3000], 0..6000 keys
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        leaf = int(rng.integers(1, 13))
        b = int(np.floor(10 ** rng.uniform(0, np.log10(3001))))
        n = int(rng.integers(0, 6001))
        out.append((leaf, max(1, b), n, 1000 + k))
    return out


@pytest.mark.parametrize("extra", [0, 1, 3, 8])
def test_random_small_configurations(rs, orc, extra):
    # 120 drawn (leaf, bucket, n) points per leaf range extra; extra 0 is the
    # minimal structure, the others the perfect, non-minimal variant
    cfgs = random_configs(120, 77 + extra)
    with cf.ThreadPoolExecutor(THREADS) as ex:
        refs = list(ex.map(lambda c: orc.build_u64(inputs.u64_keys(c[2], c[3]), c[0], c[1], extra=extra), cfgs))
    for (leaf, b, n, seed), ref in zip(cfgs, refs):
        keys = inputs.u64_keys(n, seed)
        s = (rs.Structure.build_perfect_u64(dev_u64(keys), leaf, b, extra) if extra
             else gpu_build_u64(rs, keys, leaf, b))
        assert_same_blob(s.serialize(), ref)
        if n:
            assert np.array_equal(gpu_lookup_u64(s, keys), orc.lookup_u64(ref, keys)), (leaf, b, n)


@pytest.mark.parametrize("extra", [0, 2])
def test_random_byte_string_configurations(rs, orc, extra):
    cfgs = random_configs(60, 177 + extra)
    keysets = [inputs.byte_keys(n, seed) for _, _, n, seed in cfgs]
    with cf.ThreadPoolExecutor(THREADS) as ex:
        refs = list(ex.map(lambda i: orc.build_bytes(keysets[i].data, keysets[i].offsets, cfgs[i][0], cfgs[i][1],
                                                     extra=extra), range(len(cfgs))))
    for (leaf, b, n, _), bk, ref in zip(cfgs, keysets, refs):
        data = torch.from_numpy(bk.data).cuda() if bk.data.shape[0] else torch.zeros(1, dtype=torch.uint8).cuda()
        offs = dev_u64(bk.offsets)
        s = (rs.Structure.build_perfect_bytes(data, offs, leaf, b, extra) if extra
             else rs.Structure.build_bytes(data, offs, leaf, b))
        assert_same_blob(s.serialize(), ref)
        if n:
            out = torch.empty(n, dtype=torch.int64, device="cuda")
            s.lookup_bytes(data, offs, out)
            torch.cuda.synchronize()
            assert np.array_equal(host_u64(out), orc.lookup_bytes(ref, bk.data, bk.offsets)), (leaf, b, n)


@pytest.mark.parametrize("leaf,b,n", [(8, 100, 20000), (5, 5, 3000), (3, 1, 500), (12, 40, 1500)])
def test_byte_string_structure_matches_oracle(rs, orc, leaf, b, n):
    bk = inputs.byte_keys(n, 1 + n)
    ref = orc.build_bytes(bk.data, bk.offsets, leaf, b)
    data = torch.from_numpy(bk.data).cuda()
    offs = dev_u64(bk.offsets)
    s = rs.Structure.build_bytes(data, offs, leaf, b)
    assert_same_blob(s.serialize(), ref)
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    s.lookup_bytes(data, offs, out)
    torch.cuda.synchronize()
    assert np.array_equal(host_u64(out), orc.lookup_bytes(ref, bk.data, bk.offsets))


def test_byte_strings_with_unaligned_offsets(rs, orc):
    # keys start at every byte alignment and include the empty string
    strings = [bytes([i] * i) for i in range(40)] + [b"x" * k for k in range(1, 20)]
    data = np.frombuffer(b"Z" + b"".join(strings), dtype=np.uint8)
    offs = np.zeros(len(strings) + 1, dtype=np.uint64)
    offs[0] = 1
    offs[1:] = 1 + np.cumsum([len(x) for x in strings])
    ref = orc.build_bytes(data, offs, 4, 3)
    s = rs.Structure.build_bytes(torch.from_numpy(data.copy()).cuda(), dev_u64(offs), 4, 3)
    assert_same_blob(s.serialize(), ref)


def test_long_byte_strings(rs, orc):
    # lengths 8 .. 5000 (up to 625 eight-byte words per key) at every start
    # alignment, plus the empty string; random bytes, so the keys are distinct
    rng = np.random.default_rng(31)
    lens = np.concatenate([[0, 8, 5000], rng.integers(8, 5001, 2997)]).astype(np.uint64)
    offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    data = rng.integers(0, 256, int(offsets[-1]), dtype=np.uint8)
    ref = orc.build_bytes(data, offsets, 8, 100)
    d = torch.from_numpy(data).cuda()
    o = dev_u64(offsets)
    s = rs.Structure.build_bytes(d, o, 8, 100)
    assert_same_blob(s.serialize(), ref)
    out = torch.empty(lens.shape[0], dtype=torch.int64, device="cuda")
    s.lookup_bytes(d, o, out)
    torch.cuda.synchronize()
    got = host_u64(out)
    assert np.array_equal(got, orc.lookup_bytes(ref, data, offsets))
    assert np.array_equal(np.sort(got), np.arange(lens.shape[0], dtype=np.uint64))


def test_host_buffers_give_the_same_structure(rs, orc):
    keys = inputs.u64_keys(50000, 21)
    ref = orc.build_u64(keys, 8, 100)
    s = rs.Structure.build_u64(keys, 8, 100)  # numpy: host memory
    assert_same_blob(s.serialize(), ref)
    out = np.zeros(keys.shape[0], dtype=np.uint64)
    s.lookup_u64(keys, out)  # host in, host out
    assert np.array_equal(out, orc.lookup_u64(ref, keys))
    bk = inputs.byte_keys(5000, 22)
    sb = rs.Structure.build_bytes(bk.data, bk.offsets, 8, 100)
    assert_same_blob(sb.serialize(), orc.build_bytes(bk.data, bk.offsets, 8, 100))


def test_pinned_host_buffers_are_read_in_place(rs, orc):
    # page-locked host keys are read by the signature kernel directly
    keys = inputs.u64_keys(60000, 29)
    pinned = torch.from_numpy(keys.view(np.int64)).pin_memory()
    s = rs.Structure.build_u64(pinned, 8, 100)
    assert_same_blob(s.serialize(), orc.build_u64(keys, 8, 100))
    bk = inputs.byte_keys(30000, 30)
    pd = torch.from_numpy(bk.data.copy()).pin_memory()
    po = torch.from_numpy(bk.offsets.astype(np.uint64).view(np.int64)).pin_memory()
    sb = rs.Structure.build_bytes(pd, po, 8, 100)
    assert_same_blob(sb.serialize(), orc.build_bytes(bk.data, bk.offsets, 8, 100))
    bad = bk.offsets.astype(np.uint64).copy()
    bad[11] = bad[10] - 1
    with pytest.raises(rs.RecSplitError) as e:
        rs.Structure.build_bytes(pd, torch.from_numpy(bad.view(np.int64)).pin_memory(), 8, 100)
    assert e.value.code == rs.E_INVALID


def test_serialize_round_trip(rs, orc):
    keys = inputs.u64_keys(40000, 23)
    s = gpu_build_u64(rs, keys, 5, 5)
    blob = s.serialize()
    s2 = rs.Structure.deserialize(blob)
    assert np.array_equal(s2.serialize(), blob)
    assert np.array_equal(gpu_lookup_u64(s2, keys), gpu_lookup_u64(s, keys))
    # a structure serialized by the oracle loads and answers the same
    s3 = rs.Structure.deserialize(orc.build_u64(keys, 5, 5))
    assert np.array_equal(gpu_lookup_u64(s3, keys), gpu_lookup_u64(s, keys))
    # the output range read back from the lists is n for a minimal structure
    assert s.stats()["range_size"] == s2.stats()["range_size"] == s3.stats()["range_size"] == keys.shape[0]
    assert s3.stats()["leaf_extra"] == 0


def test_repeated_keys_are_reported(rs):
    keys = inputs.u64_keys(10000, 24)
    keys[77] = keys[5000]
    with pytest.raises(rs.RecSplitError) as e:
        gpu_build_u64(rs, keys, 8, 100)
    assert e.value.code == rs.E_DUPLICATE
    # many copies that no split can place together (leaf 2)
    keys = inputs.u64_keys(300, 25)
    keys[:7] = keys[7]
    with pytest.raises(rs.RecSplitError) as e:
        gpu_build_u64(rs, keys, 2, 300)
    assert e.value.code == rs.E_DUPLICATE
    # the library stays usable afterwards
    ok = gpu_build_u64(rs, inputs.u64_keys(1000, 26), 5, 5)
    assert ok.stats()["n"] == 1000


def test_offsets_that_decrease_are_rejected(rs, orc):
    """Builds reject offsets that decrease (host and device buffers, checked
    on the device); lookups read such a key as the empty string and answer
    every other key as usual."""
    bk = inputs.byte_keys(3000, 28)
    offs = bk.offsets.astype(np.uint64)
    down = offs.copy()
    down[101] = down[100] - 1  # key 100 ends before it starts
    past = offs.copy()
    past[50] = offs[-1] + 1000  # key 49 ends past the last offset
    for bad in (down, past):
        with pytest.raises(rs.RecSplitError) as e:
            rs.Structure.build_bytes(bk.data, bad, 8, 100)
        assert e.value.code == rs.E_INVALID
        with pytest.raises(rs.RecSplitError) as e:
            rs.Structure.build_bytes(torch.from_numpy(bk.data.copy()).cuda(), dev_u64(bad), 8, 100)
        assert e.value.code == rs.E_INVALID
    s = rs.Structure.build_bytes(bk.data, offs, 8, 100)  # still usable
    assert_same_blob(s.serialize(), orc.build_bytes(bk.data, offs, 8, 100))
    data = torch.from_numpy(bk.data.copy()).cuda()
    good = torch.empty(3000, dtype=torch.int64, device="cuda")
    s.lookup_bytes(data, dev_u64(offs), good)
    got = torch.empty(3000, dtype=torch.int64, device="cuda")
    s.lookup_bytes(data, dev_u64(down), got)
    empty = torch.empty(1, dtype=torch.int64, device="cuda")
    s.lookup_bytes(torch.zeros(1, dtype=torch.uint8, device="cuda"), dev_u64(np.zeros(2, dtype=np.uint64)), empty)
    g, b = host_u64(good), host_u64(got)
    keep = np.ones(3000, dtype=bool)
    keep[[100, 101]] = False
    assert np.array_equal(b[keep], g[keep])
    assert b[100] == host_u64(empty)[0]


@pytest.mark.parametrize("extra", [0, 2])
def test_buckets_of_more_than_65536_keys(rs, orc, extra):
    # b = 65535 and n = 2b: two buckets, the larger one above 2^16 keys (65731
    # for this seed).  Its root split takes the search path that divides by
    # the part size (the fixed-point reciprocal is exact only below 2^16).
    n, b = 131070, 65535
    keys = inputs.u64_keys(n, 20)
    ref = orc.build_u64(keys, 8, b, threads=THREADS, extra=extra)
    assert orc.header(ref)["mmax"] >= 65536
    s = (rs.Structure.build_perfect_u64(dev_u64(keys), 8, b, extra) if extra
         else gpu_build_u64(rs, keys, 8, b))
    assert_same_blob(s.serialize(), ref)
    got = gpu_lookup_u64(s, keys)
    assert np.array_equal(got, orc.lookup_u64(ref, keys))
    assert np.unique(got).shape[0] == n


def test_results_do_not_depend_on_key_order(rs):
    keys = inputs.u64_keys(60000, 27)
    a = gpu_build_u64(rs, keys, 8, 100).serialize()
    b = gpu_build_u64(rs, keys[np.random.default_rng(1).permutation(keys.shape[0])], 8, 100).serialize()
    assert np.array_equal(a, b)


# ---------------------------------------------------------------- full sizes
def test_config_strings_1e7_leaf8_bucket100(rs, orc):
    """n = 10^7 random byte strings (8..32 bytes, seed 1), l = 8, b = 100:
    the whole structure byte-identical; 10^8 lookups sampled against the
    oracle; lookups of all keys a permutation of [0, n)."""
    n = 10_000_000
    bk = inputs.byte_keys(n, 1)
    data = torch.from_numpy(bk.data).cuda()
    offs = dev_u64(bk.offsets)
    # the launch shapes the benchmark times: it autotunes for this workload first
    saved = rs.recsplit_get_tuning(8)
    rs.recsplit_autotune(8, 100, n)
    try:
        s = rs.Structure.build_bytes(data, offs, 8, 100)
    finally:
        rs.recsplit_set_tuning(8, saved)
    gpu_blob = s.serialize()
    ref = orc.build_bytes(bk.data, bk.offsets, 8, 100, threads=THREADS)
    assert_same_blob(gpu_blob, ref)
    st = s.stats()
    assert abs(st["bits_per_key"] - 1.80) < 0.05

    out = torch.empty(n, dtype=torch.int64, device="cuda")
    s.lookup_bytes(data, offs, out)
    perm = torch.sort(out).values
    assert torch.equal(perm, torch.arange(n, device="cuda", dtype=torch.int64))

    q = 100_000_000
    idx = inputs.query_indices(n, q, 1)
    qdata, qoffs = inputs.device_byte_queries(bk, idx)
    qout = torch.empty(q, dtype=torch.int64, device="cuda")
    s.lookup_bytes(qdata, qoffs, qout)
    # queries are members: query j must return the index of key idx[j]
    member = out[torch.from_numpy(idx).cuda()]
    assert torch.equal(qout, member)
    sample = np.arange(0, n, 97)
    sub = inputs.gather_byte_keys(bk, sample)
    want = orc.lookup_bytes(ref, sub.data, sub.offsets)
    assert np.array_equal(host_u64(out)[sample], want)


def _oracle_buckets(orc, keys, b):
    hi, lo = orc.fingerprint_u64(keys)
    nb = -(-keys.shape[0] // b)
    bucket = (((hi >> np.uint64(32)).astype(np.float64)) * 0).astype(np.int64)
    # exact 128-bit product via the oracle's own bucket function on a vector
    bucket = np.fromiter((orc.bucket(int(h), nb) for h in hi), dtype=np.int64, count=hi.shape[0])
    return bucket, lo, nb


def test_config_u64_1e6_leaf16_bucket2000(rs, orc):
    """n = 10^6 64-bit keys (seed 2), l = 16, b = 2000 (500 buckets): sampled
    buckets rebuilt by the oracle equal the GPU's decoded indices; every
    prefix sum equals the oracle's grouping; lookups form a permutation."""
    n, leaf, b = 1_000_000, 16, 2000
    keys = inputs.u64_keys(n, 2)
    s = gpu_build_u64(rs, keys, leaf, b)
    blob = s.serialize()
    st = s.stats()
    assert abs(st["bits_per_key"] - 1.56) < 0.05
    got = gpu_lookup_u64(s, keys)
    assert np.array_equal(np.sort(got), np.arange(n, dtype=np.uint64))

    bucket, lo, nb = _oracle_buckets(orc, keys, b)
    counts = np.bincount(bucket, minlength=nb)
    prefix = np.concatenate([[0], np.cumsum(counts)])
    for i in range(0, nb + 1, 7):
        assert orc.bucket_info(blob, i)[0] == prefix[i]
    order = np.argsort(bucket, kind="stable")
    sample = [0, 137, 311, nb - 1]

    def one(bi):
        sel = lo[order[prefix[bi]:prefix[bi + 1]]]
        return orc.bucket_seeds(sel, leaf)

    with cf.ThreadPoolExecutor(len(sample)) as ex:
        seeds = list(ex.map(one, sample))
    for bi, want in zip(sample, seeds):
        assert orc.decode_bucket(blob, bi) == want, bi
    # lookups of sampled keys equal the oracle's reading of the GPU structure
    pick = np.arange(0, n, 1009)
    assert np.array_equal(got[pick], orc.lookup_u64(blob, keys[pick]))
