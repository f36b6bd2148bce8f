"""Workloads whose whole structures are checked through stored digests.

The oracle needs minutes to hours for these key sets, so
``make_oracle_digests.py`` (which calls only the oracle) builds each one once
and stores the SHA-256 of its serialized words here, beside this module.  The
GPU tests rebuild the same key sets through the C ABI and compare digests.
This module holds the case definitions (sizes, seeds, leaf and bucket sizes)
and the digest of a word array; it does no RecSplit arithmetic and imports
neither the oracle nor the library.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

# The space-optimal configuration of Table 1 (Sec. 8): 10^6 64-bit keys
# (seed 2), leaf size 16, bucket size 2000: 500 buckets.
C3 = {"n": 1_000_000, "seed": 2, "leaf": 16, "bucket": 2000}

# 4096 independent sets: sizes log-uniform in [10^3, 10^6) (seed 3), leaf and
# bucket sizes uniform over {5, 8, 12} x {5, 100, 2000}.
C4 = {"count": 4096, "lo": 1000, "hi": 1_000_000, "seed": 3}

# Table 2 scale: 10^9 64-bit keys (seed 4), leaf size 8, bucket size 100.
BIG = {"n": 1_000_000_000, "seed": 4, "leaf": 8, "bucket": 100}

# Leaves of the largest sizes (Sec. 5.4 bounds leaves by 24): one bucket of
# 3l + 1 keys (seed 100 + l), whose root split has parts l, l, l, 1.
LARGE_LEAVES = [{"leaf": l, "n": 3 * l + 1, "bucket": 3 * l + 1, "seed": 100 + l} for l in (22, 23, 24)]

# The (leaf, bucket) sweep of the space and construction-time figures of
# Sec. 8: 64-bit keys (seed 4), the first n of the stream for each leaf size.
SWEEP_BUCKETS = (5, 100, 2000)
SWEEP_SEED = 4


def sweep_n(leaf: int) -> int:
    """Keys per sweep point: fewer as the leaf searches grow (about e times
    the work per unit of leaf size)."""
    if leaf <= 12:
        return 1_000_000
    if leaf <= 14:
        return 200_000
    if leaf <= 16:
        return 50_000
    if leaf <= 18:
        return 10_000
    return {19: 2000, 20: 1000, 21: 500}[leaf]


SWEEP_LEAVES = tuple(range(2, 22))


def sweep_points():
    return [(l, b, sweep_n(l)) for l in SWEEP_LEAVES for b in SWEEP_BUCKETS]


def words_digest(words: np.ndarray) -> str:
    """SHA-256 (hex) of a structure's serialized 64-bit words, little endian."""
    return hashlib.sha256(np.ascontiguousarray(words, dtype="<u8").tobytes()).hexdigest()


def bucket_digest(s: int, o: int, seeds) -> str:
    """Short digest of one bucket: its prefix sum s_i, bit offset o_i and the
    indices of its tree in preorder."""
    w = np.array([s, o, len(seeds), *seeds], dtype="<u8")
    return hashlib.sha256(w.tobytes()).hexdigest()[:16]


def path(name: str) -> str:
    return os.path.join(HERE, name)


def load(name: str):
    """A stored digest file, or None if it has not been generated."""
    p = path(name)
    if not os.path.exists(p):
        return None
    with open(p) as f:
        return json.load(f)
