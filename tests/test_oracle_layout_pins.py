"""The serialized layout, rebuilt in this file from its definition.

Sec. 6.2 stores a bucket's splitting-tree indices as Golomb-Rice codes, all
fixed parts in preorder and then all unary parts in preorder; Sec. 6.3 and
Sec. 7.4 store the bucket prefix sums and bit offsets as a double Elias-Fano
list with a two-level inventory.  The byte-level choices the paper leaves
open are the readings R12-R16 (bit order, code conventions, beta, the
minimum-delta rescale, lower widths, inventory spacing and 0xFFFF entries).

Here the whole structure is written again by plain Python integer code that
follows those definitions, from pieces the other pins already tie to the
paper: the signature and bucket functions, the splitting strategy (Sec. 5.4),
the Golomb-Rice parameters (Eq. gr) and the first successful index of every
node (brute force).  The oracle's own writer and readers are not used: the
result must equal the oracle's structure word for word, so a wrong bit order,
a swapped section, an off-by-one in a unary code or in an inventory entry
anywhere in the oracle fails here.
"""
import numpy as np
import pytest

from paper_1910_06416_gb300 import inputs

MAGIC = int.from_bytes(b"RECSPLT1", "little")
M64 = (1 << 64) - 1


class Bits:
    """A bit array as a Python int: bit k of the array is bit k of the int
    (bit k mod 64 of 64-bit word k / 64, R12)."""

    def __init__(self):
        self.v = 0

    def put(self, pos, value, width):
        assert 0 <= value < (1 << width) or width == 0
        self.v |= value << pos

    def words(self, nbits):
        nw = (nbits + 63) // 64
        return [(self.v >> (64 * k)) & M64 for k in range(nw)]


def preorder(orc, leaf, m):
    """Node sizes of the splitting tree of m keys in preorder (sizes >= 2
    carry a code; Sec. 4, Sec. 5.4)."""
    if m <= 1:
        return []
    parts = orc.strategy(leaf, m)
    out = [m]
    for p in parts:
        out += preorder(orc, leaf, p)
    return out


def lg(x):
    return x.bit_length() - 1


def structure_from_definitions(orc, keys, leaf, b):
    n = len(keys)
    hi, lo = orc.fingerprint_u64(keys)
    N = -(-n // b)
    bucket = [(int(h) * N) >> 64 for h in hi]  # fixed-point inversion (Sec. 6.1)
    members = [[] for _ in range(N)]
    for j, bk in enumerate(bucket):
        members[bk].append(int(lo[j]))
    sizes = [len(x) for x in members]
    s = [0]
    for m in sizes:
        s.append(s[-1] + m)

    # Sec. 6.2: per bucket, the fixed parts (low r bits of each index, least
    # significant bit first) in preorder, then the unary parts (q zeros, then
    # a one) in preorder, the bucket's code starting at o_i (R12, R13)
    tree = Bits()
    o = [0]
    codes = 0
    for i in range(N):
        m = sizes[i]
        nodes = preorder(orc, leaf, m)
        seeds = orc.bucket_seeds(np.array(members[i], dtype=np.uint64), leaf) if m >= 2 else []
        assert len(seeds) == len(nodes)
        codes += len(nodes)
        pos = o[-1]
        rs_ = [orc.golomb_rice(leaf, k) for k in nodes]
        for r, x in zip(rs_, seeds):
            tree.put(pos, x & ((1 << r) - 1), r)
            pos += r
        for r, x in zip(rs_, seeds):
            pos += x >> r
            tree.put(pos, 1, 1)
            pos += 1
        o.append(pos)
    T = o[-1]

    # Sec. 6.3 / 7.4 with R14-R16: beta = floor(T 2^32 / n), beta s_i =
    # floor(s_i beta / 2^32); each list rescaled by its smallest gap delta
    # (stored y_i = x_i - i delta), lower width max(0, floor(lg(y_N / (N+1)))),
    # one bit at (y_i >> L) + i in the upper bits
    beta = (T << 32) // n if n else 0
    xa = s[:]
    xb = [o[i] - ((s[i] * beta) >> 32) for i in range(N + 1)]

    def rescale(x):
        d = min(x[i + 1] - x[i] for i in range(N)) if N else 0
        return d, [x[i] - i * d for i in range(N + 1)]

    da, ya = rescale(xa)
    db, yb = rescale(xb)

    def width(u):
        q = u // (N + 1)
        return lg(q) if q else 0

    la, lb = width(ya[-1]), width(yb[-1])
    lower, upa, upb = Bits(), Bits(), Bits()
    pa, pb = [], []
    for i in range(N + 1):
        lower.put(i * (la + lb), ya[i] & ((1 << la) - 1), la)
        lower.put(i * (la + lb) + la, yb[i] & ((1 << lb) - 1), lb)
        pa.append((ya[i] >> la) + i)
        pb.append((yb[i] >> lb) + i)
        upa.put(pa[-1], 1, 1)
        upb.put(pb[-1], 1, 1)
    ua, ub = pa[-1] + 1, pb[-1] + 1
    # inventory: the position of every 2^14-th one as a 64-bit anchor, and of
    # every 2^8-th one as a 16-bit offset from its anchor (0xFFFF if it does
    # not fit); the two lists interleaved
    anchors = []
    for k in range(N // (1 << 14) + 1):
        anchors += [pa[k << 14], pb[k << 14]]
    subs = []
    for j in range(N // (1 << 8) + 1):
        i, k = j << 8, j >> 6
        for p, anchor in ((pa, anchors[2 * k]), (pb, anchors[2 * k + 1])):
            d = p[i] - anchor
            subs.append(d if d < 0xFFFF else 0xFFFF)
    if len(subs) % 4:
        subs += [0] * (4 - len(subs) % 4)
    sub_words = [sum(subs[4 * w + t] << (16 * t) for t in range(4)) for w in range(len(subs) // 4)]

    body = (tree.words(T) + lower.words((N + 1) * (la + lb)) + upa.words(ua) + upb.words(ub) + anchors
            + sub_words)
    header = [MAGIC, n, leaf, b, N, T, max(sizes) if N else 0, beta, da & M64, db & M64, la, lb, ua, ub,
              16 + len(body), codes]
    return np.array(header + body, dtype=np.uint64)


@pytest.mark.parametrize("leaf,b,n,seed", [(2, 4, 40, 1), (5, 5, 300, 2), (4, 9, 200, 3), (8, 100, 2500, 4),
                                           (3, 1, 30, 5), (6, 1000, 1500, 6), (8, 100, 0, 7), (8, 100, 1, 8),
                                           (1, 3, 50, 9)])
def test_structure_equals_its_definition(orc, leaf, b, n, seed):
    keys = inputs.u64_keys(n, seed)
    want = structure_from_definitions(orc, keys, leaf, b)
    got = orc.build_u64(keys, leaf, b)
    assert got.shape == want.shape, (got.shape, want.shape)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, f"{bad.size} words differ, first at {bad[:6].tolist()}"


def test_small_bucket_codes_by_hand(orc):
    """One bucket of 4 keys with leaf size 2 (split 2 + 2, then two leaves):
    three codes in preorder [root, left leaf, right leaf]; the bits are
    r_root + r_2 + r_2 fixed bits, then three unary codes."""
    keys = inputs.u64_keys(4, 11)
    blob = structure_from_definitions(orc, keys, 2, 4)
    hi, lo = orc.fingerprint_u64(keys)
    seeds = orc.bucket_seeds(lo, 2)
    assert orc.strategy(2, 4) == [2, 2] and len(seeds) == 3
    r4, r2 = orc.golomb_rice(2, 4), orc.golomb_rice(2, 2)
    fixed = [(seeds[0], r4), (seeds[1], r2), (seeds[2], r2)]
    bits = []
    for x, r in fixed:
        bits += [(x >> k) & 1 for k in range(r)]
    for x, r in fixed:
        bits += [0] * (x >> r) + [1]
    T = int(blob[5])
    assert T == len(bits)
    word = 0
    for k, bit in enumerate(bits):
        word |= bit << k
    got = 0
    for k in range((T + 63) // 64):
        got |= int(blob[16 + k]) << (64 * k)
    assert got == word
    assert np.array_equal(orc.build_u64(keys, 2, 4), blob)
