"""Every leaf size from 13 to 21 against the oracle, word for word.

The search kernel for full leaves is compiled once per leaf size (Sec. 5.2:
the bijection test of l keys); each size here runs on key sets whose buckets
produce full l-key leaves, with the phased test (the default from l = 10:
two phases up to 12 keys, three phases with per-warp survivor queues from
13) and with the one-phase test, and the structures must equal the oracle's.
Sizes 22 to 24 take the oracle minutes per leaf and are checked against
stored oracle digests (test_gpu_digests.py).
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def key_sets(leaf):
    """(n, bucket, seed): buckets of about 2l keys (one full leaf each, split
    l + rest) and, up to l = 17, buckets of about 5l keys (root splits of
    fanout 5, four or five full leaves each)."""
    out = [(6 * leaf + 5, 2 * leaf + 1, 200 + leaf)]
    if leaf <= 17:
        out.append((30 * leaf, 5 * leaf, 300 + leaf))
    return out


@pytest.mark.parametrize("leaf", list(range(13, 22)))
def test_full_leaves_of_every_size_match_oracle(rs, orc, leaf):
    sets = key_sets(leaf)
    keys = [inputs.u64_keys(n, sd) for n, _, sd in sets]
    with cf.ThreadPoolExecutor(len(sets)) as ex:
        refs = list(ex.map(lambda i: orc.build_u64(keys[i], leaf, sets[i][1], threads=THREADS), range(len(sets))))
    for i, ((n, b, _), ref) in enumerate(zip(sets, refs)):
        assert orc.header(ref)["codes"] > 0
    saved = rs.recsplit_get_tuning(leaf)
    try:
        for two_phase in (1, 0):
            rs.recsplit_set_tuning(leaf, dict(saved, leaf_two_phase=two_phase,
                                              leaf_seeds_per_lane=4 if two_phase else 1))
            for (n, b, _), k, ref in zip(sets, keys, refs):
                s = rs.Structure.build_u64(dev(k), leaf, b)
                got = s.serialize()
                assert np.array_equal(got, ref), (leaf, n, b, two_phase)
                out = torch.empty(n, dtype=torch.int64, device="cuda")
                s.lookup_u64(dev(k), out)
                torch.cuda.synchronize()
                assert np.array_equal(out.cpu().numpy().view(np.uint64), orc.lookup_u64(ref, k))
    finally:
        rs.recsplit_set_tuning(leaf, saved)
