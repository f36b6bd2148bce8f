"""Whole structures of the large workloads against stored oracle digests.

The oracle takes minutes to hours on these key sets, so the committed script
``tests/golden/make_oracle_digests.py`` (which calls only ``oracle/``) built
each once and stored the SHA-256 of its serialized words.  Here the CUDA
path builds the same key sets through the C ABI and every structure's digest
must match: the whole of every structure is then identical to the oracle's.

 - the space-optimal configuration of Table 1 (10^6 keys, l = 16, b = 2000),
   with a per-bucket digest to locate a difference;
 - all 4096 sets of the batched configuration, in one batched build;
 - leaves of 22, 23 and 24 keys (Sec. 5.4 bounds leaves by 24);
 - every point of the (l, b) sweep, l = 2..21, b in {5, 100, 2000};
 - 10^9 keys at l = 8, b = 100 (the scale of Table 2).
"""
import os
import sys

import numpy as np
import pytest

from paper_1910_06416_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import digest_cases as D  # noqa: E402


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1910_06416_gb300 import build
    build.build()
    import paper_1910_06416_gb300.recsplit as rs
    rs.lib()
    return rs


def stored(name):
    data = D.load(f"oracle_digests_{name}.json")
    assert data is not None, f"tests/golden/oracle_digests_{name}.json is missing"
    return data


def dev_keys(n, seed):
    return inputs.device_splitmix64(seed, n)


def first_bad_bucket(orc, blob, digests):
    for i, want in enumerate(digests):
        s, o = orc.bucket_info(blob, i)
        if D.bucket_digest(s, o, orc.decode_bucket(blob, i)) != want:
            return i
    return None


def test_space_optimal_configuration_whole_structure(rs, orc):
    ref = stored("c3")
    c = D.C3
    s = rs.Structure.build_u64(dev_keys(c["n"], c["seed"]), c["leaf"], c["bucket"])
    blob = s.serialize()
    if D.words_digest(blob) != ref["sha256"]:
        bad = first_bad_bucket(orc, blob, ref["bucket_digests"])
        raise AssertionError(f"structure differs from the oracle's ({blob.shape[0]} words, oracle "
                             f"{ref['words']}); first differing bucket: {bad}")
    assert abs(s.stats()["bits_per_key"] - 1.56) < 0.05  # Table 1


def test_batched_configuration_every_set(rs):
    ref = stored("c4")
    c = D.C4
    plan = inputs.batch_sets(c["count"], c["lo"], c["hi"], c["seed"])
    assert len(plan) == ref["sets"]
    keys = [dev_keys(n, sd) for n, _, _, sd in plan]
    hs = rs.recsplit_build_batch([(k, l, b) for k, (n, l, b, _) in zip(keys, plan)])
    try:
        bad = []
        for i, h in enumerate(hs):
            if D.words_digest(rs.recsplit_serialize(h))[:16] != ref["set_sha256_16"][i]:
                bad.append(i)
        assert not bad, f"{len(bad)} sets differ from the oracle's, first {bad[:5]} {[plan[i] for i in bad[:3]]}"
    finally:
        for h in hs:
            rs.recsplit_free(h)


def test_leaves_of_22_to_24_keys(rs, orc):
    ref = stored("leaves")
    for c in ref["cases"]:
        keys = inputs.u64_keys(c["n"], c["seed"])
        s = rs.Structure.build_u64(keys, c["leaf"], c["bucket"])
        blob = s.serialize()
        assert orc.decode_bucket(blob, 0) == c["seeds"], c["leaf"]
        assert D.words_digest(blob) == c["sha256"], c["leaf"]
        got = np.zeros(c["n"], dtype=np.uint64)
        s.lookup_u64(keys, got)
        assert np.array_equal(np.sort(got), np.arange(c["n"], dtype=np.uint64))


def test_sweep_points(rs):
    ref = stored("sweep")
    assert ref["seed"] == D.SWEEP_SEED
    bad = []
    keys = {}
    for p in ref["points"]:
        n = p["n"]
        if n not in keys:
            keys.clear()
            keys[n] = dev_keys(n, D.SWEEP_SEED)
        s = rs.Structure.build_u64(keys[n], p["leaf"], p["bucket"])
        if D.words_digest(s.serialize()) != p["sha256"]:
            bad.append((p["leaf"], p["bucket"], n))
        s.free()
    assert not bad, f"sweep points that differ from the oracle: {bad}"


def test_table2_scale_billion_keys(rs):
    ref = stored("big")
    c = D.BIG
    keys = dev_keys(c["n"], c["seed"])
    s = rs.Structure.build_u64(keys, c["leaf"], c["bucket"])
    del keys
    torch.cuda.empty_cache()
    blob = s.serialize()
    assert blob.shape[0] == ref["words"]
    assert D.words_digest(blob) == ref["sha256"]
