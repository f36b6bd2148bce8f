"""recsplit_deserialize checks every part of a structure that steers a
lookup's reads (Sec. 6.2 codes, Sec. 6.3 / 7.4 lists and inventories)
before loading it.  Damaged structures are rejected on the host with
RECSPLIT_E_INVALID; an intact one passes the check and only then needs the
device (without a GPU the load fails later, with another code)."""
import numpy as np
import pytest

from paper_1910_06416_gb300 import inputs


@pytest.fixture(scope="module")
def rs():
    from paper_1910_06416_gb300 import build
    build.build()
    import paper_1910_06416_gb300.recsplit as rs
    rs.lib()
    return rs


def _load(rs, words):
    """None if the structure check passed (the load may still fail on the
    device side), else the message of the rejection."""
    try:
        h = rs.recsplit_deserialize(words)
    except rs.RecSplitError as e:
        if e.code == rs.E_INVALID:
            return str(e)
        return None
    rs.recsplit_free(h)
    return None


@pytest.fixture(scope="module")
def blob(orc):
    keys = inputs.u64_keys(30000, 61)
    return orc.build_u64(keys, 8, 100)


def _flip(words, bit):
    w = words.copy()
    w[bit >> 6] ^= np.uint64(1 << (bit & 63))
    return w


def test_intact_structures_pass(rs, orc, blob):
    assert _load(rs, blob) is None
    for leaf, b, n, extra in [(5, 5, 2000, 0), (8, 100, 1, 0), (8, 100, 0, 0), (12, 9, 3000, 2), (3, 1000, 5000, 1)]:
        words = orc.build_u64(inputs.u64_keys(n, 62), leaf, b, extra=extra)
        assert _load(rs, words) is None, (leaf, b, n, extra)


def test_unary_bits_are_checked(rs, orc, blob):
    lay = orc.layout(blob)
    h = orc.header(blob)
    # the first bucket with a code: flip a bit of its unary part
    for i in range(h["nbuckets"]):
        s0, o0 = orc.bucket_info(blob, i)
        s1, o1 = orc.bucket_info(blob, i + 1)
        if s1 - s0 >= 2:
            break
    fixed, _ = orc.skip(8, s1 - s0)
    for bit in (o0 + fixed, o1 - 1, (o0 + fixed + o1) // 2):
        msg = _load(rs, _flip(blob, 64 * lay["tree"] + bit))
        assert msg and "structure check failed" in msg, bit


def test_fixed_bits_are_not_steering(rs, orc, blob):
    # a fixed part only changes an index, and a lookup then moves to another
    # child of the same node: reads stay inside the bucket, the check passes
    lay = orc.layout(blob)
    assert _load(rs, _flip(blob, 64 * lay["tree"] + 0)) is None


def test_lists_and_inventories_are_checked(rs, orc, blob):
    lay = orc.layout(blob)
    h = orc.header(blob)
    cases = {
        "upper bits A": 64 * lay["upper_a"] + 3,
        "upper bits B": 64 * lay["upper_b"] + 5,
        "anchor": 64 * lay["anchors"] + 1,
        "u16 offset": 64 * lay["subs"] + 16 * 2 + 1,  # second offset of list A
        "lower bits of B": 64 * lay["lower"] + h["low_a"] + h["low_b"] + h["low_a"] + max(0, h["low_b"] - 1),
    }
    for name, bit in cases.items():
        msg = _load(rs, _flip(blob, bit))
        assert msg and "structure check failed" in msg, name


def test_header_fields_are_checked(rs, blob):
    for field, delta in ((6, 1), (15, 1), (5, 1)):  # largest bucket, codes, tree bits
        w = blob.copy()
        w[field] += np.uint64(delta)
        assert _load(rs, w), field


def test_inventory_overflow_entries_pass(rs, orc):
    # a 16-bit offset of 0xFFFF makes select fall back to an earlier entry of
    # its anchor's block: accepted anywhere but at a block's first entry
    blob = orc.build_u64(inputs.u64_keys(90000, 3), 5, 5)
    lay = orc.layout(blob)
    w = blob.copy()
    subs = w[lay["subs"]:].view(np.uint16)
    for e in (2 * 3, 2 * 3 + 1, 2 * 70, 2 * 65 + 1, 2 * 66 + 1):
        subs[e] = 0xFFFF
    assert _load(rs, w) is None
    for e in (0, 2 * 64 + 1):  # first entries of the blocks of anchors 0 and 1
        w = blob.copy()
        w[lay["subs"]:].view(np.uint16)[e] = 0xFFFF
        assert _load(rs, w), e
