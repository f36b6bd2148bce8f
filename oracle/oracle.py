"""ctypes binding of the RecSplit oracle -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this module.  It compiles ``recsplit_oracle.c`` with the
host C compiler into ``oracle/_lib/`` on first use and wraps its functions in
numpy-friendly calls.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "recsplit_oracle.c")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "liboracle.so")

E_INVALID, E_DUPLICATE, E_SEARCH_LIMIT, E_NOMEM = -1, -2, -4, -5
HEADER_FIELDS = ("magic", "n", "leaf", "bucket_size", "nbuckets", "tree_bits", "mmax", "beta",
                 "delta_a", "delta_b", "low_a", "low_b", "upper_a_bits", "upper_b_bits", "words", "codes")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into a shared object (idempotent)."""
    os.makedirs(LIBDIR, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-shared", "-fPIC",
                               "-o", tmp, SRC, "-lm", "-lpthread"])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            u64, u32, i64, p = C.c_uint64, C.c_uint32, C.c_int64, C.c_void_p
            L.orc_mix64.restype = u64
            L.orc_mix64.argtypes = [u64]
            L.orc_phi.restype = u32
            L.orc_phi.argtypes = [u64, u32, u64, u64]
            L.orc_bucket.restype = u64
            L.orc_bucket.argtypes = [u64, u64]
            L.orc_strategy.restype = C.c_int
            L.orc_strategy.argtypes = [u32, u64, p, p, C.c_int]
            L.orc_log_success.restype = C.c_double
            L.orc_log_success.argtypes = [u32, u64]
            L.orc_log_success_e.restype = C.c_double
            L.orc_log_success_e.argtypes = [u32, u32, u64]
            L.orc_golomb_rice_x_e.restype = C.c_double
            L.orc_golomb_rice_x_e.argtypes = [u32, u32, u64]
            L.orc_golomb_rice_e.restype = C.c_int
            L.orc_golomb_rice_e.argtypes = [u32, u32, u64]
            L.orc_node_range.restype = u64
            L.orc_node_range.argtypes = [u32, u32, u64]
            L.orc_leaf_seed_range.restype = i64
            L.orc_leaf_seed_range.argtypes = [p, u64, u64, u32, u64]
            L.orc_build_u64_e.restype = C.c_int
            L.orc_build_u64_e.argtypes = [p, u64, u32, u32, u32, C.c_int, p, p]
            L.orc_build_bytes_e.restype = C.c_int
            L.orc_build_bytes_e.argtypes = [p, p, u64, u32, u32, u32, C.c_int, p, p]
            L.orc_build_fingerprints_e.restype = C.c_int
            L.orc_build_fingerprints_e.argtypes = [p, p, u64, u32, u32, u32, C.c_int, p, p]
            L.orc_bucket_seeds_from_keys_e.restype = C.c_int
            L.orc_bucket_seeds_from_keys_e.argtypes = [p, u64, u32, u32, p, p]
            L.orc_golomb_rice_x.restype = C.c_double
            L.orc_golomb_rice_x.argtypes = [u32, u64]
            L.orc_golomb_rice.restype = C.c_int
            L.orc_golomb_rice.argtypes = [u32, u64]
            L.orc_skip.restype = C.c_int
            L.orc_skip.argtypes = [u32, u64, p, p]
            L.orc_leaf_seed.restype = i64
            L.orc_leaf_seed.argtypes = [p, u64, u32, u64]
            L.orc_split_seed.restype = i64
            L.orc_split_seed.argtypes = [p, u64, u32, u32, u64]
            L.orc_fingerprint_u64.argtypes = [p, u64, p, p]
            L.orc_fingerprint_bytes.argtypes = [p, p, u64, p, p]
            L.orc_build_fingerprints.restype = C.c_int
            L.orc_build_fingerprints.argtypes = [p, p, u64, u32, u32, C.c_int, p, p]
            L.orc_build_u64.restype = C.c_int
            L.orc_build_u64.argtypes = [p, u64, u32, u32, C.c_int, p, p]
            L.orc_build_bytes.restype = C.c_int
            L.orc_build_bytes.argtypes = [p, p, u64, u32, u32, C.c_int, p, p]
            L.orc_free.argtypes = [p]
            L.orc_lookup_u64.restype = C.c_int
            L.orc_lookup_u64.argtypes = [p, p, u64, p]
            L.orc_lookup_bytes.restype = C.c_int
            L.orc_lookup_bytes.argtypes = [p, p, p, u64, p]
            L.orc_lookup_fingerprints.restype = C.c_int
            L.orc_lookup_fingerprints.argtypes = [p, p, p, u64, p]
            L.orc_bucket_info.restype = C.c_int
            L.orc_bucket_info.argtypes = [p, u64, p, p]
            L.orc_decode_bucket.restype = C.c_int
            L.orc_decode_bucket.argtypes = [p, u64, p, u64, p]
            L.orc_bucket_seeds_from_keys.restype = C.c_int
            L.orc_bucket_seeds_from_keys.argtypes = [p, u64, u32, p, p]
            L.orc_select_linear.restype = u64
            L.orc_select_linear.argtypes = [p, C.c_int, u64]
            L.orc_select_inventory.restype = u64
            L.orc_select_inventory.argtypes = [p, C.c_int, u64]
            L.orc_layout_words.argtypes = [p, p]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle error {code}")
        self.code = code


def _check(rc: int):
    if rc != 0:
        raise OracleError(rc)


# ---------------------------------------------------------------- pieces
def mix64(z: int) -> int:
    return int(lib().orc_mix64(z))


def phi(lo: int, depth: int, index: int, m: int) -> int:
    return int(lib().orc_phi(lo, depth, index, m))


def bucket(hi: int, nbuckets: int) -> int:
    return int(lib().orc_bucket(hi, nbuckets))


def strategy(leaf: int, m: int) -> list[int]:
    """Part sizes of a node with m keys ([] for a leaf)."""
    parts = np.zeros(64, dtype=np.uint64)
    unit = np.zeros(1, dtype=np.uint64)
    f = lib().orc_strategy(leaf, m, _ptr(unit), _ptr(parts), 64)
    assert f >= 0
    return [int(x) for x in parts[:f]]


def log_success(leaf: int, m: int, extra: int = 0) -> float:
    """ln of one trial's success probability at a node of m keys (leaf
    range m + extra for leaves)."""
    if extra:
        return float(lib().orc_log_success_e(leaf, extra, m))
    return float(lib().orc_log_success(leaf, m))


def golomb_rice(leaf: int, m: int, extra: int = 0) -> int:
    if extra:
        return int(lib().orc_golomb_rice_e(leaf, extra, m))
    return int(lib().orc_golomb_rice(leaf, m))


def golomb_rice_x(leaf: int, m: int, extra: int = 0) -> float:
    if extra:
        return float(lib().orc_golomb_rice_x_e(leaf, extra, m))
    return float(lib().orc_golomb_rice_x(leaf, m))


def node_range(leaf: int, extra: int, m: int) -> int:
    """Output range of the subtree of a node of m keys."""
    return int(lib().orc_node_range(leaf, extra, m))


def skip(leaf: int, m: int) -> tuple[int, int]:
    fb = np.zeros(1, dtype=np.uint64)
    nc = np.zeros(1, dtype=np.uint64)
    _check(lib().orc_skip(leaf, m, _ptr(fb), _ptr(nc)))
    return int(fb[0]), int(nc[0])


def leaf_seed(lo: np.ndarray, depth: int = 0, cap: int = 1 << 36, range_size: int | None = None) -> int:
    """First index whose values on the leaf's keys are distinct in
    [0, range_size) (default: the number of keys, a bijection)."""
    lo = np.ascontiguousarray(lo, dtype=np.uint64)
    if range_size is not None:
        return int(lib().orc_leaf_seed_range(_ptr(lo), lo.shape[0], range_size, depth, cap))
    return int(lib().orc_leaf_seed(_ptr(lo), lo.shape[0], depth, cap))


def split_seed(lo: np.ndarray, leaf: int, depth: int = 0, cap: int = 1 << 36) -> int:
    lo = np.ascontiguousarray(lo, dtype=np.uint64)
    return int(lib().orc_split_seed(_ptr(lo), lo.shape[0], depth, leaf, cap))


def fingerprint_u64(keys: np.ndarray):
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    hi = np.empty_like(keys)
    lo = np.empty_like(keys)
    lib().orc_fingerprint_u64(_ptr(keys), keys.shape[0], _ptr(hi), _ptr(lo))
    return hi, lo


def fingerprint_bytes(data: np.ndarray, offsets: np.ndarray):
    data = np.ascontiguousarray(data, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    n = offsets.shape[0] - 1
    hi = np.empty(n, dtype=np.uint64)
    lo = np.empty(n, dtype=np.uint64)
    lib().orc_fingerprint_bytes(_ptr(data), _ptr(offsets), n, _ptr(hi), _ptr(lo))
    return hi, lo


# ---------------------------------------------------------------- build
def _take_blob(blobp: C.c_void_p, words: np.ndarray) -> np.ndarray:
    nw = int(words[0])
    arr = np.ctypeslib.as_array(C.cast(blobp, C.POINTER(C.c_uint64)), shape=(nw,)).copy()
    lib().orc_free(blobp)
    return arr


def build_fingerprints(hi, lo, leaf: int, bucket_size: int, threads: int = 1, extra: int = 0) -> np.ndarray:
    hi = np.ascontiguousarray(hi, dtype=np.uint64)
    lo = np.ascontiguousarray(lo, dtype=np.uint64)
    blobp, words = C.c_void_p(), np.zeros(1, dtype=np.uint64)
    _check(lib().orc_build_fingerprints_e(_ptr(hi), _ptr(lo), hi.shape[0], leaf, extra, bucket_size, threads,
                                          C.byref(blobp), _ptr(words)))
    return _take_blob(blobp, words)


def build_u64(keys: np.ndarray, leaf: int, bucket_size: int, threads: int = 1, extra: int = 0) -> np.ndarray:
    """Serialized structure (uint64 words) for 64-bit keys; extra > 0 builds
    the perfect, non-minimal variant (leaf ranges m + extra)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    blobp, words = C.c_void_p(), np.zeros(1, dtype=np.uint64)
    if extra:
        _check(lib().orc_build_u64_e(_ptr(keys), keys.shape[0], leaf, extra, bucket_size, threads,
                                     C.byref(blobp), _ptr(words)))
    else:
        _check(lib().orc_build_u64(_ptr(keys), keys.shape[0], leaf, bucket_size, threads, C.byref(blobp),
                                   _ptr(words)))
    return _take_blob(blobp, words)


def build_bytes(data: np.ndarray, offsets: np.ndarray, leaf: int, bucket_size: int,
                threads: int = 1, extra: int = 0) -> np.ndarray:
    data = np.ascontiguousarray(data, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    blobp, words = C.c_void_p(), np.zeros(1, dtype=np.uint64)
    if extra:
        _check(lib().orc_build_bytes_e(_ptr(data), _ptr(offsets), offsets.shape[0] - 1, leaf, extra,
                                       bucket_size, threads, C.byref(blobp), _ptr(words)))
    else:
        _check(lib().orc_build_bytes(_ptr(data), _ptr(offsets), offsets.shape[0] - 1, leaf, bucket_size,
                                     threads, C.byref(blobp), _ptr(words)))
    return _take_blob(blobp, words)


# ---------------------------------------------------------------- read
def header(blob: np.ndarray) -> dict:
    h = {k: int(blob[i]) for i, k in enumerate(HEADER_FIELDS)}
    h["leaf_extra"] = (h["leaf"] >> 8) & 0xFF  # word 2: leaf size | leaf range extra << 8
    h["leaf"] &= 0xFF
    for k in ("delta_a", "delta_b"):
        if h[k] >= 1 << 63:
            h[k] -= 1 << 64
    return h


def lookup_u64(blob: np.ndarray, keys: np.ndarray) -> np.ndarray:
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    out = np.empty(keys.shape[0], dtype=np.uint64)
    _check(lib().orc_lookup_u64(_ptr(blob), _ptr(keys), keys.shape[0], _ptr(out)))
    return out


def lookup_bytes(blob: np.ndarray, data: np.ndarray, offsets: np.ndarray) -> np.ndarray:
    data = np.ascontiguousarray(data, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    out = np.empty(offsets.shape[0] - 1, dtype=np.uint64)
    _check(lib().orc_lookup_bytes(_ptr(blob), _ptr(data), _ptr(offsets), out.shape[0], _ptr(out)))
    return out


def lookup_fingerprints(blob: np.ndarray, hi: np.ndarray, lo: np.ndarray) -> np.ndarray:
    hi = np.ascontiguousarray(hi, dtype=np.uint64)
    lo = np.ascontiguousarray(lo, dtype=np.uint64)
    out = np.empty(hi.shape[0], dtype=np.uint64)
    _check(lib().orc_lookup_fingerprints(_ptr(blob), _ptr(hi), _ptr(lo), hi.shape[0], _ptr(out)))
    return out


def bucket_info(blob: np.ndarray, i: int) -> tuple[int, int]:
    """(s_i, o_i): keys before bucket i and bit offset of bucket i."""
    s = np.zeros(1, dtype=np.uint64)
    o = np.zeros(1, dtype=np.uint64)
    _check(lib().orc_bucket_info(_ptr(blob), i, _ptr(s), _ptr(o)))
    return int(s[0]), int(o[0])


def decode_bucket(blob: np.ndarray, b: int) -> list[int]:
    """Indices of bucket b in preorder, read back from the bit array."""
    cap = 1 << 16
    seeds = np.zeros(cap, dtype=np.uint64)
    cnt = np.zeros(1, dtype=np.uint64)
    _check(lib().orc_decode_bucket(_ptr(blob), b, _ptr(seeds), cap, _ptr(cnt)))
    return [int(x) for x in seeds[:int(cnt[0])]]


def bucket_seeds(lo: np.ndarray, leaf: int, extra: int = 0) -> list[int]:
    """Preorder indices of the tree of one bucket whose keys have lower halves `lo`."""
    lo = np.ascontiguousarray(lo, dtype=np.uint64)
    seeds = np.zeros(max(1, lo.shape[0]), dtype=np.uint64)
    cnt = np.zeros(1, dtype=np.uint64)
    _check(lib().orc_bucket_seeds_from_keys_e(_ptr(lo), lo.shape[0], leaf, extra, _ptr(seeds), _ptr(cnt)))
    return [int(x) for x in seeds[:int(cnt[0])]]


def select_linear(blob, lst: int, rank: int) -> int:
    return int(lib().orc_select_linear(_ptr(blob), lst, rank))


def select_inventory(blob, lst: int, rank: int) -> int:
    return int(lib().orc_select_inventory(_ptr(blob), lst, rank))


def layout(blob) -> dict:
    out = np.zeros(7, dtype=np.uint64)
    lib().orc_layout_words(_ptr(blob), _ptr(out))
    return dict(zip(("tree", "lower", "upper_a", "upper_b", "anchors", "subs", "total"),
                    (int(x) for x in out)))


def bits_per_key(blob: np.ndarray) -> float:
    h = header(blob)
    return 64.0 * blob.shape[0] / max(1, h["n"])


def tree_bits_per_key(blob: np.ndarray) -> float:
    h = header(blob)
    return h["tree_bits"] / max(1, h["n"])
