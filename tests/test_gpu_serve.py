"""Serving engine: builds and lookups of different sizes submitted while
others run; every result must equal the same request served alone."""
import time

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


def _slice(keys, a, b):
    offs = keys.offsets[a:b + 1] - keys.offsets[a]
    return inputs.ByteKeys(keys.data[int(keys.offsets[a]):int(keys.offsets[b])].copy(), offs.copy())


def _wait_all(rs, srv, ids, timeout=120.0):
    got = {}
    t0 = time.time()
    while len(got) < len(ids) and time.time() - t0 < timeout:
        for c in rs.recsplit_server_poll(srv, 256, wait_ms=50):
            got[c["request_id"]] = c
    assert len(got) == len(ids)
    return got


def test_mixed_requests_equal_their_results_alone(rs):
    pool = inputs.byte_keys(600000, 5)
    sizes = inputs.log_uniform_sizes(24, 1000, 60000, 7)
    srv = rs.recsplit_server_create(hbm_budget_bytes=8 << 30)
    try:
        builds, pos = [], 0
        for n in sizes:
            kb = _slice(pool, pos, pos + int(n))
            pos += int(n)
            rid = rs.recsplit_server_submit_build_bytes(srv, kb.data, kb.offsets, 8, 100)
            builds.append((rid, kb))
        # one request with a repeated key: only it fails
        bad_keys = inputs.u64_keys(400, 9)
        bad_keys[5] = bad_keys[7]
        bad_id = rs.recsplit_server_submit_build_u64(srv, bad_keys, 5, 5)
        done = _wait_all(rs, srv, [b[0] for b in builds] + [bad_id])
        assert done[bad_id]["status"] == rs.E_DUPLICATE
        # lookups of mixed sizes against the resident structures, submitted together
        lookups = []
        rng = np.random.default_rng(3)
        for rid, kb in builds:
            assert done[rid]["status"] == 0
            q = int(rng.integers(1, 5000))
            idx = rng.integers(0, kb.n, q)
            qk = inputs.gather_byte_keys(kb, idx)
            out = np.zeros(q, dtype=np.uint64)
            lid = rs.recsplit_server_submit_lookup_bytes(srv, rid, qk.data, qk.offsets, out)
            lookups.append((lid, rid, kb, qk, out))
        # a build arriving while lookups run
        late = _slice(pool, pos + 1000, pos + 21000)
        late_id = rs.recsplit_server_submit_build_bytes(srv, late.data, late.offsets, 8, 100)
        done2 = _wait_all(rs, srv, [l[0] for l in lookups] + [late_id])
        for lid, rid, kb, qk, out in lookups:
            assert done2[lid]["status"] == 0
            alone = rs.Structure.build_bytes(kb.data, kb.offsets, 8, 100)
            assert np.array_equal(rs.recsplit_serialize(rs.recsplit_server_structure(srv, rid)), alone.serialize())
            want = np.zeros(qk.n, dtype=np.uint64)
            alone.lookup_bytes(qk.data, qk.offsets, want)
            assert np.array_equal(out, want)
        assert done2[late_id]["status"] == 0
        st = rs.recsplit_server_stats(srv)
        assert st["resident_structures"] == len(builds) + 1
        batched = [c for c in list(done.values()) + list(done2.values()) if c["batch_size"] > 1]
        assert batched, "no request was served together with another"
        for rid, _ in builds:
            rs.recsplit_server_release(srv, rid)
        assert rs.recsplit_server_stats(srv)["resident_structures"] == 1
    finally:
        rs.recsplit_server_destroy(srv)


def test_memory_budget_admission(rs):
    keys = inputs.u64_keys(200000, 21)
    srv = rs.recsplit_server_create(hbm_budget_bytes=25 << 20)  # fits one 200k build at a time
    try:
        ids = [rs.recsplit_server_submit_build_u64(srv, keys, 8, 100) for _ in range(3)]
        big = inputs.u64_keys(2_000_000, 22)
        big_id = rs.recsplit_server_submit_build_u64(srv, big, 8, 100)  # never fits
        done = _wait_all(rs, srv, ids + [big_id])
        assert all(done[i]["status"] == 0 for i in ids)
        assert all(done[i]["batch_size"] == 1 for i in ids)
        assert done[big_id]["status"] == rs.E_NOMEM
        blobs = [rs.recsplit_serialize(rs.recsplit_server_structure(srv, i)) for i in ids]
        assert all(np.array_equal(b, blobs[0]) for b in blobs)
    finally:
        rs.recsplit_server_destroy(srv)


def test_short_build_overtakes_a_long_one(rs):
    """A 10^4-key build submitted while a long build runs (10^6 keys, l = 16,
    b = 2000, about a second) is taken by a free build worker at once and
    completes first; both structures equal the same builds served alone."""
    big = inputs.u64_keys(1_000_000, 2)
    small = inputs.byte_keys(10_000, 41)
    srv = rs.recsplit_server_create(hbm_budget_bytes=8 << 30)
    try:
        big_id = rs.recsplit_server_submit_build_u64(srv, big, 16, 2000)
        t0 = time.time()
        while rs.recsplit_server_stats(srv)["in_flight_bytes"] == 0 and time.time() - t0 < 10:
            time.sleep(0.001)
        time.sleep(0.05)  # the long build is on the device
        small_id = rs.recsplit_server_submit_build_bytes(srv, small.data, small.offsets, 8, 100)
        order = []
        got = {}
        while len(got) < 2 and time.time() - t0 < 120:
            for c in rs.recsplit_server_poll(srv, 16, wait_ms=20):
                got[c["request_id"]] = c
                order.append(c["request_id"])
        assert order == [small_id, big_id], order
        assert got[small_id]["status"] == 0 and got[big_id]["status"] == 0
        assert got[small_id]["batch_size"] == 1
        assert got[small_id]["queue_ms"] < 100
        alone_small = rs.Structure.build_bytes(small.data, small.offsets, 8, 100)
        assert np.array_equal(rs.recsplit_serialize(rs.recsplit_server_structure(srv, small_id)),
                              alone_small.serialize())
        alone_big = rs.Structure.build_u64(big, 16, 2000)
        assert np.array_equal(rs.recsplit_serialize(rs.recsplit_server_structure(srv, big_id)),
                              alone_big.serialize())
    finally:
        rs.recsplit_server_destroy(srv)
