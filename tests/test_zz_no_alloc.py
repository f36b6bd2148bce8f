"""The allocation-free lookup entry point (recsplit_lookup_u64_static).

It serves callers that cannot allocate device memory while answering
lookups; its results must equal those of recsplit_lookup_u64 on the same
structure, call after call, since both run the same lookup and every value
is an exact integer.  This file is collected last so that a failure here
cannot stop the other tests of a run.
"""
import concurrent.futures as cf

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


def test_static_lookup_equals_allocating_lookup_twice(rs, orc):
    keys = inputs.u64_keys(200000, 31)
    s = rs.Structure.build_u64(torch.from_numpy(keys.view(np.int64)).cuda(), 8, 100)
    ref = orc.build_u64(keys, 8, 100)
    members = keys[inputs.query_indices(keys.shape[0], 300000, 32)]
    others = inputs.splitmix64(33, 50000)
    for q in (members, others, members[:rs.STATIC_LOOKUP_MAX]):
        want = np.zeros(q.shape[0], dtype=np.uint64)
        rs.recsplit_lookup_u64(s.handle, q, want)
        # and directly against the oracle's lookup on its own structure
        assert np.array_equal(want, orc.lookup_u64(ref, q))
        for _ in range(2):  # two calls in a row share the staging array
            got = np.full(q.shape[0], 7, dtype=np.uint64)
            rs.recsplit_lookup_u64_static(s.handle, q, got)
            assert np.array_equal(got, want)
    # device buffers work too
    d_q = torch.from_numpy(members.view(np.int64)).cuda()
    d_out = torch.empty_like(d_q)
    rs.recsplit_lookup_u64_static(s.handle, d_q, d_out)
    want = np.zeros(members.shape[0], dtype=np.uint64)
    rs.recsplit_lookup_u64(s.handle, members, want)
    assert np.array_equal(d_out.cpu().numpy().view(np.uint64), want)


def test_static_lookup_rejects_oversized_batches(rs):
    keys = inputs.u64_keys(1000, 34)
    s = rs.Structure.build_u64(keys, 5, 5)
    big = np.zeros(rs.STATIC_LOOKUP_MAX + 1, dtype=np.uint64)
    out = np.zeros_like(big)
    with pytest.raises(rs.RecSplitError) as e:
        rs.recsplit_lookup_u64_static(s.handle, big, out)
    assert e.value.code == rs.E_INVALID


def test_static_lookups_from_several_host_threads(rs):
    # the calls share one staging array; the library runs them one at a time,
    # so every thread gets the results of its own keys
    keys = inputs.u64_keys(100000, 35)
    s = rs.Structure.build_u64(torch.from_numpy(keys.view(np.int64)).cuda(), 8, 100)
    qs = [keys[inputs.query_indices(keys.shape[0], 200000 + 1000 * t, 36 + t)] for t in range(8)]
    wants = []
    for q in qs:
        w = np.zeros(q.shape[0], dtype=np.uint64)
        rs.recsplit_lookup_u64(s.handle, q, w)
        wants.append(w)

    def run(t):
        got = np.zeros(qs[t].shape[0], dtype=np.uint64)
        for _ in range(3):
            rs.recsplit_lookup_u64_static(s.handle, qs[t], got)
            if not np.array_equal(got, wants[t]):
                return False
        return True

    with cf.ThreadPoolExecutor(8) as ex:
        assert all(ex.map(run, range(8)))


def test_static_lookup_makes_no_device_allocation(rs, orc):
    # the next device allocation of the library on this thread is made to
    # fail (on the host, as if the device were out of memory): the
    # allocation-free lookup must still succeed, while an allocating lookup
    # that decodes the bucket lists per batch fails
    keys = inputs.u64_keys(50000, 37)
    s = rs.Structure.build_u64(keys, 8, 100)
    q = keys[inputs.query_indices(keys.shape[0], 20000, 38)]
    want = orc.lookup_u64(orc.build_u64(keys, 8, 100), q)
    rs.recsplit_inject_alloc_failure(0)
    try:
        for _ in range(2):
            got = np.zeros(q.shape[0], dtype=np.uint64)
            rs.recsplit_lookup_u64_static(s.handle, q, got)
            assert np.array_equal(got, want)
        # still armed: the allocating lookup with host buffers stages them in
        # device memory it allocates, and fails
        with pytest.raises(rs.RecSplitError) as e:
            rs.recsplit_lookup_u64(s.handle, q, np.zeros(q.shape[0], dtype=np.uint64))
        assert e.value.code == rs.E_NOMEM
    finally:
        rs.recsplit_inject_alloc_failure(-1)
