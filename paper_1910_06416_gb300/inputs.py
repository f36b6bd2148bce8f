"""Seeded synthetic key sets and query streams.

Both the CUDA path and the oracle draw their inputs from here.  The module
holds only the input recipe -- the splitmix64 pseudo-random stream (Steele,
Lea, Flood 2014) and how its outputs become keys -- and none of RecSplit's
arithmetic.  Everything is numpy on the host; the optional device helpers
use torch only to move and gather bytes.

Recipe (stated once, used everywhere):

* ``splitmix64(seed)`` output number k (k = 0, 1, ...) is the splitmix64
  finalizer applied to ``seed + (k + 1) * 0x9E3779B97F4A7C15`` (mod 2^64).
* 64-bit keys with seed s: outputs 0 .. n-1 of ``splitmix64(s)``.  The state
  walk is a permutation and the finalizer a bijection, so they are distinct.
* Byte-string keys with seed s: key i has length ``8 + floor(A_i * 25 / 2^64)``
  (uniform in 8..32) with A = ``splitmix64(s)``, and its bytes are the
  little-endian bytes of outputs 4i .. 4i+3 of ``splitmix64(s ^ BYTES_SALT)``,
  cut to that length.  Distinctness is checked (the first 8 bytes are one
  full random word).
* Queries drawn from a key set with seed s: query j is key
  ``floor(Q_j * n / 2^64)`` with Q = ``splitmix64(s ^ QUERY_SALT)``.
"""
from __future__ import annotations

import numpy as np

WEYL = np.uint64(0x9E3779B97F4A7C15)
BYTES_SALT = 0xA5A5A5A5A5A5A5A5
QUERY_SALT = 0x5851F42D4C957F2D
MASK32 = np.uint64(0xFFFFFFFF)


def _finalize(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= np.uint64(0xBF58476D1CE4E5B9)
    z ^= z >> np.uint64(27)
    z *= np.uint64(0x94D049BB133111EB)
    z ^= z >> np.uint64(31)
    return z


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+count-1 of the splitmix64 stream seeded with `seed`."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * WEYL
    return _finalize(state)


def _mulhi_small(x: np.ndarray, m: int) -> np.ndarray:
    """floor(x * m / 2^64) for uint64 x and 0 < m < 2^32, exactly."""
    assert 0 < m < (1 << 32)
    mm = np.uint64(m)
    hi = x >> np.uint64(32)
    lo = x & MASK32
    t = lo * mm
    t = hi * mm + (t >> np.uint64(32))
    return t >> np.uint64(32)


def _mulhi(x: np.ndarray, m: int) -> np.ndarray:
    """floor(x * m / 2^64) for uint64 x and 0 < m < 2^64, exactly."""
    if m < (1 << 32):
        return _mulhi_small(x, m)
    m_hi, m_lo = np.uint64(m >> 32), np.uint64(m & 0xFFFFFFFF)
    x_hi, x_lo = x >> np.uint64(32), x & MASK32
    ll = x_lo * m_lo
    lh = x_lo * m_hi
    hl = x_hi * m_lo
    hh = x_hi * m_hi
    mid = (ll >> np.uint64(32)) + (lh & MASK32) + (hl & MASK32)
    return hh + (lh >> np.uint64(32)) + (hl >> np.uint64(32)) + (mid >> np.uint64(32))


def u64_keys(n: int, seed: int) -> np.ndarray:
    """n distinct 64-bit keys, uniform, from splitmix64(seed)."""
    return splitmix64(seed, n)


class ByteKeys:
    """Packed byte strings: key i is ``data[offsets[i]:offsets[i+1]]``."""

    def __init__(self, data: np.ndarray, offsets: np.ndarray):
        self.data = data
        self.offsets = offsets

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    def key(self, i: int) -> bytes:
        return self.data[self.offsets[i]:self.offsets[i + 1]].tobytes()


def byte_keys(n: int, seed: int, check_distinct: bool = True) -> ByteKeys:
    """n distinct random byte strings of length uniform in 8..32."""
    lengths = (np.uint64(8) + _mulhi_small(splitmix64(seed, n), 25)).astype(np.int64)
    words = splitmix64(seed ^ BYTES_SALT, 4 * n)
    padded = words.view(np.uint8).reshape(n, 32)  # little-endian byte order
    offsets = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(lengths, out=offsets[1:])
    mask = np.arange(32)[None, :] < lengths[:, None]
    data = padded[mask]
    if check_distinct and n > 1:
        first = words[0::4]
        if np.unique(first).shape[0] != n:
            raise RuntimeError("byte-string generator produced a repeated first word")
    return ByteKeys(np.ascontiguousarray(data), offsets)


def query_indices(n: int, count: int, seed: int) -> np.ndarray:
    """Indices (uniform with replacement) of `count` queries into a key set of n."""
    return _mulhi(splitmix64(seed ^ QUERY_SALT, count), n).astype(np.int64)


def gather_byte_keys(keys: ByteKeys, idx: np.ndarray) -> ByteKeys:
    """Packed byte strings of keys[idx] (host)."""
    lengths = keys.lengths().astype(np.int64)[idx]
    offsets = np.zeros(idx.shape[0] + 1, dtype=np.uint64)
    np.cumsum(lengths, out=offsets[1:])
    starts = keys.offsets[:-1].astype(np.int64)[idx]
    total = int(offsets[-1])
    pos = np.arange(total, dtype=np.int64) - np.repeat(offsets[:-1].astype(np.int64), lengths)
    src = np.repeat(starts, lengths) + pos
    return ByteKeys(keys.data[src], offsets)


def log_uniform_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """`count` sizes floor(10^U) with U uniform in [log10 lo, log10 hi) (53-bit draws)."""
    u = (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    a, b = np.log10(lo), np.log10(hi)
    return np.floor(10.0 ** (a + (b - a) * u)).astype(np.int64)


# ----------------------------------------------------------------------
# Device helpers (torch as plumbing only).
# ----------------------------------------------------------------------

def device_byte_queries(keys: ByteKeys, idx: np.ndarray, device="cuda"):
    """Packed query strings keys[idx] materialised on `device`.

    Returns (data uint8 tensor, offsets int64 tensor of len q+1).  Done with
    a fixed 32-byte padded view of the key set so that 10^8 queries gather
    in one pass on the device.
    """
    import torch

    n = keys.n
    lengths = torch.from_numpy(keys.lengths().astype(np.int64)).to(device)
    starts = torch.from_numpy(keys.offsets[:-1].astype(np.int64)).to(device)
    data = torch.from_numpy(keys.data).to(device)
    col = torch.arange(32, device=device, dtype=torch.int64)
    src = (starts[:, None] + col[None, :]).clamp_(max=max(int(data.shape[0]) - 1, 0))
    padded = data[src] if data.numel() else torch.zeros((n, 32), dtype=torch.uint8, device=device)
    del src
    qi = torch.from_numpy(idx).to(device)
    qlen = lengths[qi]
    offsets = torch.zeros(qi.shape[0] + 1, dtype=torch.int64, device=device)
    torch.cumsum(qlen, 0, out=offsets[1:])
    out = torch.empty(int(offsets[-1].item()), dtype=torch.uint8, device=device)
    chunk = 1 << 24
    for c0 in range(0, qi.shape[0], chunk):
        c1 = min(qi.shape[0], c0 + chunk)
        rows = padded[qi[c0:c1]]
        mask = col[None, :] < qlen[c0:c1, None]
        out[int(offsets[c0].item()):int(offsets[c1].item())] = rows[mask]
    return out, offsets


def device_splitmix64(seed: int, count: int, start: int = 0, device="cuda"):
    """splitmix64(seed) outputs start .. start+count-1 computed on `device`
    (int64 tensor holding the same bits as splitmix64()).  torch has no
    unsigned 64-bit arithmetic, so logical right shifts are masked."""
    import torch

    def u2s(x):
        return x - (1 << 64) if x >= 1 << 63 else x

    k = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    z = k * u2s(int(WEYL)) + u2s(seed & 0xFFFFFFFFFFFFFFFF)

    def shr(x, s):
        return (x >> s) & ((1 << (64 - s)) - 1)

    z = z ^ shr(z, 30)
    z = z * u2s(0xBF58476D1CE4E5B9)
    z = z ^ shr(z, 27)
    z = z * u2s(0x94D049BB133111EB)
    return z ^ shr(z, 31)


def batch_sets(count: int, lo: int, hi: int, seed: int, leaves=(5, 8, 12), buckets=(5, 100, 2000)):
    """The key-set plan of a batch: per set its size (log-uniform in
    [lo, hi)), its (leaf, bucket) pair (uniform over the product of `leaves`
    and `buckets`), and the seed of its keys.  Set i's 64-bit keys are
    u64_keys(size_i, seed_i)."""
    sizes = log_uniform_sizes(count, lo, hi, seed)
    pick = _mulhi_small(splitmix64(seed ^ 0x243F6A8885A308D3, count), len(leaves) * len(buckets)).astype(np.int64)
    combos = [(l, b) for l in leaves for b in buckets]
    seeds = splitmix64(seed ^ 0x13198A2E03707344, count)
    return [(int(sizes[i]), combos[int(pick[i])][0], combos[int(pick[i])][1], int(seeds[i])) for i in range(count)]
