"""Batched construction (many structures of uneven sizes and mixed leaf and
bucket sizes in one pass) and batched lookup, against the oracle and against
one-at-a-time builds."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def test_device_generator_equals_host_generator():
    got = inputs.device_splitmix64(77, 100000, start=5).cpu().numpy().view(np.uint64)
    assert np.array_equal(got, inputs.splitmix64(77, 100000, start=5))


def test_small_batch_matches_oracle_and_single_builds(rs, orc):
    plan = inputs.batch_sets(48, 1000, 30000, 3)
    plan += [(0, 5, 5, 1), (1, 8, 100, 2), (2, 12, 9, 3), (17, 8, 2000, 4)]  # degenerate sets
    keys = [inputs.u64_keys(n, sd) for n, _, _, sd in plan]
    dkeys = [dev(k) for k in keys]
    hs = rs.recsplit_build_batch([(dk, l, b) for dk, (n, l, b, _) in zip(dkeys, plan)])
    try:
        blobs = [rs.recsplit_serialize(h) for h in hs]

        def ref(i):
            n, l, b, _ = plan[i]
            return orc.build_u64(keys[i], l, b, threads=2)

        with cf.ThreadPoolExecutor(THREADS) as ex:
            refs = list(ex.map(ref, range(len(plan))))
        for i, (blob, r) in enumerate(zip(blobs, refs)):
            assert np.array_equal(blob, r), (i, plan[i])
        for i in range(0, len(plan), 7):
            n, l, b, _ = plan[i]
            single = rs.Structure.build_u64(dkeys[i], l, b)
            assert np.array_equal(single.serialize(), blobs[i])
        # batched lookup over all structures equals per-structure lookups
        rng = np.random.default_rng(5)
        ids = rng.integers(0, len(plan), 200000).astype(np.uint32)
        qk = np.array([keys[i][rng.integers(0, max(1, keys[i].shape[0]))] if keys[i].shape[0] else 0
                       for i in ids], dtype=np.uint64)
        out = torch.empty(ids.shape[0], dtype=torch.int64, device="cuda")
        rs.recsplit_lookup_batch(hs, torch.from_numpy(ids.view(np.int32)).cuda(), dev(qk), out)
        got = out.cpu().numpy().view(np.uint64)
        for i in range(len(plan)):
            sel = ids == i
            if sel.any():
                assert np.array_equal(got[sel], orc.lookup_u64(refs[i], qk[sel])), i
        # host buffers too
        hout = np.zeros(ids.shape[0], dtype=np.uint64)
        rs.recsplit_lookup_batch(hs, ids, qk, hout)
        assert np.array_equal(hout, got)
        # the batch above has more queries than the structures have buckets
        # (lists decoded once); a small batch selects in the lists per query
        buckets = sum(-(-n // b) + 1 for n, _, b, _ in plan if n)
        few = 1000
        assert few < buckets <= ids.shape[0] - len(plan)
        out_few = torch.empty(few, dtype=torch.int64, device="cuda")
        rs.recsplit_lookup_batch(hs, torch.from_numpy(ids[:few].view(np.int32)).cuda(), dev(qk[:few]), out_few)
        assert np.array_equal(out_few.cpu().numpy().view(np.uint64), got[:few])
    finally:
        for h in hs:
            rs.recsplit_free(h)


def test_batched_lookup_with_structure_ids_out_of_range(rs, orc):
    # ids not below the number of structures give 2^64 - 1 and read nothing;
    # the other queries are unaffected (device and host buffers, with and
    # without the per-batch decode of the lists)
    keys = [inputs.u64_keys(3000, 41), inputs.u64_keys(5000, 42)]
    refs = [orc.build_u64(keys[0], 5, 5), orc.build_u64(keys[1], 8, 100)]
    hs = [rs.Structure.build_u64(dev(keys[0]), 5, 5), rs.Structure.build_u64(dev(keys[1]), 8, 100)]
    rng = np.random.default_rng(43)
    for q in (50, 20000):
        ids = rng.integers(0, 4, q).astype(np.uint32)
        ids[:3] = [2, 0xFFFFFFFF, 1]
        qk = np.array([keys[i % 2][rng.integers(0, keys[i % 2].shape[0])] for i in ids], dtype=np.uint64)
        want = np.full(q, np.iinfo(np.uint64).max, dtype=np.uint64)
        for i in (0, 1):
            sel = ids == i
            want[sel] = orc.lookup_u64(refs[i], qk[sel])
        out = torch.empty(q, dtype=torch.int64, device="cuda")
        rs.recsplit_lookup_batch([h.handle for h in hs], torch.from_numpy(ids.view(np.int32)).cuda(), dev(qk), out)
        assert np.array_equal(out.cpu().numpy().view(np.uint64), want)
        hout = np.zeros(q, dtype=np.uint64)
        rs.recsplit_lookup_batch([h.handle for h in hs], ids, qk, hout)
        assert np.array_equal(hout, want)


def test_batch_mixing_byte_string_and_u64_sets(rs, orc):
    # 40 sets: 64-bit keys or byte strings, leaf sizes {3, 5, 8, 12}, leaf
    # range extras {0, 2} (8 parameter classes), 0..20000 keys each
    rng = np.random.default_rng(51)
    plan = []
    for i in range(40):
        plan.append((int(rng.integers(0, 20001)) if i % 9 else int(rng.integers(0, 3)),
                     int(rng.choice([3, 5, 8, 12])), int(rng.choice([5, 9, 100, 1000])), int(rng.choice([0, 2])),
                     bool(rng.integers(0, 2)), 500 + i))
    data, sets = [], []
    for n, leaf, b, e, is_bytes, seed in plan:
        if is_bytes:
            bk = inputs.byte_keys(n, seed)
            d = torch.from_numpy(bk.data).cuda() if bk.data.shape[0] else torch.zeros(1, dtype=torch.uint8).cuda()
            data.append(bk)
            sets.append((d, dev(bk.offsets), leaf, b, {"leaf_extra": e}))
        else:
            k = inputs.u64_keys(n, seed)
            data.append(k)
            sets.append((dev(k), leaf, b, {"leaf_extra": e}))

    def ref(i):
        n, leaf, b, e, is_bytes, _ = plan[i]
        if is_bytes:
            return orc.build_bytes(data[i].data, data[i].offsets, leaf, b, threads=2, extra=e)
        return orc.build_u64(data[i], leaf, b, threads=2, extra=e)

    with cf.ThreadPoolExecutor(THREADS) as ex:
        refs = list(ex.map(ref, range(len(plan))))
    hs = rs.recsplit_build_batch(sets)
    try:
        for i, h in enumerate(hs):
            assert np.array_equal(rs.recsplit_serialize(h), refs[i]), plan[i]
    finally:
        for h in hs:
            rs.recsplit_free(h)


def test_batch_structures_outlive_each_other(rs, orc):
    plan = [(5000, 5, 5, 11), (7000, 8, 100, 12)]
    keys = [inputs.u64_keys(n, sd) for n, _, _, sd in plan]
    hs = rs.recsplit_build_batch([(dev(k), l, b) for k, (n, l, b, _) in zip(keys, plan)])
    rs.recsplit_free(hs[0])  # the arena stays alive for the other
    out = np.zeros(keys[1].shape[0], dtype=np.uint64)
    rs.recsplit_lookup_u64(hs[1], keys[1], out)
    assert np.array_equal(out, orc.lookup_u64(orc.build_u64(keys[1], 8, 100), keys[1]))
    rs.recsplit_free(hs[1])


def test_batch_4096_sets_full_size(rs, orc):
    """4096 sets, sizes log-uniform in [10^3, 10^6) (seed 3), leaf sizes
    {5, 8, 12} x bucket sizes {5, 100, 2000}: every set's lookups form a
    permutation; sampled sets equal the oracle; 10^9 batched lookups agree
    with per-set lookups on a sample."""
    plan = inputs.batch_sets(4096, 1000, 1000000, 3)
    total = sum(p[0] for p in plan)
    keys = [inputs.device_splitmix64(sd, n) for n, _, _, sd in plan]
    hs = rs.recsplit_build_batch([(k, l, b) for k, (n, l, b, _) in zip(keys, plan)])
    try:
        # permutation per set: all member lookups, shifted by the set's base
        base = 0
        got_all = torch.empty(total, dtype=torch.int64, device="cuda")
        for i, (n, l, b, _) in enumerate(plan):
            out = got_all[base:base + n]
            rs.recsplit_lookup_u64(hs[i], keys[i], out)
            out += base
            base += n
        assert torch.equal(torch.sort(got_all).values, torch.arange(total, device="cuda"))
        del got_all
        # sampled sets against the oracle (smallest of each parameter pair)
        best = {}
        for i, (n, l, b, _) in enumerate(plan):
            if (l, b) not in best or n < plan[best[(l, b)]][0]:
                best[(l, b)] = i
        for i in best.values():
            n, l, b, sd = plan[i]
            ref = orc.build_u64(inputs.u64_keys(n, sd), l, b, threads=THREADS)
            assert np.array_equal(rs.recsplit_serialize(hs[i]), ref), plan[i]
        # 10^9 batched lookups, in chunks
        q = 1_000_000_000
        chunk = 100_000_000
        sizes = torch.tensor([p[0] for p in plan], device="cuda", dtype=torch.int64)
        flat = torch.cat(keys)
        offs = torch.zeros(len(plan) + 1, dtype=torch.int64, device="cuda")
        torch.cumsum(sizes, 0, out=offs[1:])
        checked = 0
        for c0 in range(0, q, chunk):
            r = inputs.device_splitmix64(0xC4C4, 2 * chunk, start=2 * c0)
            ids = ((r[0::2] >> 1) % len(plan)).to(torch.int32)
            pos = (r[1::2] >> 1) % sizes[ids.long()]
            qk = flat[offs[ids.long()] + pos]
            out = torch.empty(chunk, dtype=torch.int64, device="cuda")
            rs.recsplit_lookup_batch(hs, ids, qk, out)
            if c0 == 0:
                for i in range(0, len(plan), 512):
                    sel = (ids == i).nonzero().flatten()[:1000]
                    if sel.numel():
                        want = torch.empty(sel.numel(), dtype=torch.int64, device="cuda")
                        rs.recsplit_lookup_u64(hs[i], qk[sel].contiguous(), want)
                        assert torch.equal(out[sel], want)
                        checked += sel.numel()
            del qk, out, ids, pos, r
        del flat
        assert checked > 0
    finally:
        for h in hs:
            rs.recsplit_free(h)
