"""Pins of the oracle's perfect, non-minimal variant (leaf range extra e > 0).

The paper's conclusion notes that enlarging the codomain of the bijections
gives compact perfect, non-minimal hash functions, and leaves the details
open.  The reading pinned here: a leaf of m >= 2 keys maps its keys
injectively into [0, m + e); splits are unchanged; a subtree's output range is
the sum of its leaves' ranges; buckets are laid out one after another by
their ranges.  Every expected value below comes from a definition, an
enumeration or a brute force, not from the oracle's own formulas.
"""
import itertools
import math
from fractions import Fraction
from functools import lru_cache

import numpy as np
import pytest

from paper_1910_06416_gb300 import inputs


@pytest.mark.parametrize("m,R", [(2, 3), (3, 4), (3, 6), (4, 5), (4, 7), (5, 6), (2, 9)])
def test_injection_probability_by_enumeration(orc, m, R):
    good = sum(1 for f in itertools.product(range(R), repeat=m) if len(set(f)) == m)
    p = Fraction(good, R ** m)
    leaf = max(m, 2)
    assert math.isclose(orc.log_success(leaf, m, extra=R - m), math.log(p), rel_tol=1e-12, abs_tol=1e-12)


def test_zero_extra_is_the_minimal_structure(orc):
    keys = inputs.u64_keys(20000, 40)
    assert np.array_equal(orc.build_u64(keys, 8, 100, extra=0), orc.build_u64(keys, 8, 100))


def test_leaf_seed_is_first_injection(orc):
    rng = np.random.default_rng(41)
    for trial in range(60):
        m = int(rng.integers(2, 8))
        R = m + int(rng.integers(1, 5))
        depth = int(rng.integers(0, 5))
        lo = rng.integers(0, 1 << 63, size=m, dtype=np.int64).astype(np.uint64)
        i = orc.leaf_seed(lo, depth, range_size=R)
        distinct = lambda j: len({orc.phi(int(x), depth, j, R) for x in lo}) == m
        assert distinct(i)
        assert not any(distinct(j) for j in range(i))


@pytest.mark.parametrize("leaf,extra", [(5, 1), (8, 2), (8, 8), (12, 3), (16, 4)])
def test_node_range_is_size_plus_extra_per_coded_leaf(orc, leaf, extra):
    @lru_cache(None)
    def coded_leaves(m):
        if m <= 1:
            return 0
        if m <= leaf:
            return 1
        return sum(coded_leaves(k) for k in orc.strategy(leaf, m))
    prev = -1
    for m in list(range(0, 300)) + [1000, 2000, 2345]:
        r = orc.node_range(leaf, extra, m)
        assert r == m + extra * coded_leaves(m), (m, r)
        if m < 300:
            assert r > prev  # strictly increasing: a bucket's size is read back from its range
            prev = r


@pytest.mark.parametrize("leaf,b,extra,n", [(5, 5, 1, 30000), (8, 100, 2, 60000), (8, 100, 8, 40000),
                                            (12, 9, 4, 5000), (16, 40, 6, 800), (3, 1000, 2, 5000)])
def test_perfect_hash_into_the_range(orc, leaf, b, extra, n):
    keys = inputs.u64_keys(n, 42)
    blob = orc.build_u64(keys, leaf, b, threads=4, extra=extra)
    h = orc.header(blob)
    assert h["leaf"] == leaf and h["leaf_extra"] == extra
    out = orc.lookup_u64(blob, keys)
    # output range: the bucket sizes under the bucket function, each bucket
    # contributing the range of its tree
    hi, _ = orc.fingerprint_u64(keys)
    nb = -(-n // b)
    sizes = np.bincount([orc.bucket(int(x), nb) for x in hi], minlength=nb)
    total = sum(orc.node_range(leaf, extra, int(m)) for m in sizes)
    assert np.unique(out).shape[0] == n  # injective
    assert int(out.max()) < total
    # and every bucket's keys land in that bucket's own slice of the range
    starts = np.concatenate([[0], np.cumsum([orc.node_range(leaf, extra, int(m)) for m in sizes])])
    bk = np.array([orc.bucket(int(x), nb) for x in hi])
    assert np.all((out >= starts[bk]) & (out < starts[bk + 1]))


def test_decoded_seeds_equal_per_bucket_search(orc):
    keys = inputs.u64_keys(20000, 43)
    leaf, b, extra = 8, 100, 3
    blob = orc.build_u64(keys, leaf, b, extra=extra)
    hi, lo = orc.fingerprint_u64(keys)
    nb = -(-keys.shape[0] // b)
    bk = np.array([orc.bucket(int(x), nb) for x in hi])
    for bucket in range(0, nb, 17):
        want = orc.bucket_seeds(lo[bk == bucket], leaf, extra=extra)
        assert orc.decode_bucket(blob, bucket) == want


@pytest.mark.parametrize("kind,m,R,samples", [("leaf", 8, 10, 800), ("leaf", 5, 7, 3000)])
def test_injection_seeds_are_geometric(orc, kind, m, R, samples):
    # indices of the first injection over random key sets: Geometric(p) with
    # p counted by enumeration of the value tuples' distinctness (Monte Carlo
    # free: p = R!/((R-m)! R^m) is the fraction of injective tuples)
    p = math.perm(R, m) / R ** m
    rng = np.random.default_rng(44)
    seeds = [orc.leaf_seed(rng.integers(0, 1 << 63, size=m, dtype=np.int64).astype(np.uint64), 0, range_size=R)
             for _ in range(samples)]
    mean = float(np.mean(seeds)) + 1
    sd = math.sqrt((1 - p) / p ** 2 / samples)
    assert abs(mean - 1 / p) < 5 * sd, (mean, 1 / p)


def test_extra_lowers_tree_bits_and_leaf_trials(orc):
    keys = inputs.u64_keys(200000, 45)
    t0 = orc.tree_bits_per_key(orc.build_u64(keys, 8, 100, threads=8))
    t2 = orc.tree_bits_per_key(orc.build_u64(keys, 8, 100, threads=8, extra=2))
    assert t2 < t0 - 0.2  # leaf seeds need ~lg(1/p) bits; p grows 7.5-fold at R = 10


def test_invalid_extra_is_rejected(orc):
    keys = inputs.u64_keys(100, 46)
    with pytest.raises(Exception):
        orc.build_u64(keys, 24, 10, extra=9)  # leaf + extra must be at most 32


@pytest.mark.parametrize("leaf,extra", [(5, 1), (8, 2), (12, 4), (16, 8)])
def test_leaf_golomb_rice_minimises_expected_length(orc, leaf, extra):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    golden = (1 + mpmath.sqrt(5)) / 2
    for m in range(2, leaf + 1):
        R = m + extra
        p = mpmath.mpf(math.perm(R, m)) / mpmath.mpf(R) ** m
        lens = []
        for r in range(48):
            q = mpmath.power(1 - p, 2 ** r)
            lens.append(r + 1 + q / (1 - q))
        best = min(range(48), key=lambda r: lens[r])
        assert orc.golomb_rice(leaf, m, extra=extra) == best, (m, R)
        # Sec. 5.4: with r > 0 the expected unary length lies in [phi, 1 + phi]
        # (with r = 0, for p near 1, it can be shorter)
        assert lens[best] - best <= 1 + golden + 1e-12
        if best > 0:
            assert lens[best] - best >= golden - 1e-12
