"""Thin ctypes binding of the C ABI in ``include/recsplit.h``.

The functions carry the C names and only marshal arguments: every step of
construction and lookup runs in the CUDA library.  Arrays may be torch
tensors (CUDA or CPU) or numpy arrays; their data pointers are passed as
they are and the library copies host buffers itself.  Loading fails loudly
if the compiled library is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "librecsplit.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "recsplit.h")

OK = 0
E_INVALID, E_DUPLICATE, E_SEARCH_LIMIT, E_NOMEM, E_CUDA, E_TIMEOUT = -1, -2, -4, -5, -6, -7

_lock = threading.Lock()
_lib = None


class Stats(C.Structure):
    _fields_ = [("n", C.c_uint64), ("leaf_size", C.c_uint32), ("bucket_size", C.c_uint32),
                ("num_buckets", C.c_uint64), ("tree_bits", C.c_uint64), ("total_bits", C.c_uint64),
                ("max_bucket", C.c_uint64), ("num_codes", C.c_uint64), ("tree_bits_per_key", C.c_double),
                ("bits_per_key", C.c_double), ("leaf_extra", C.c_uint32), ("reserved", C.c_uint32),
                ("range_size", C.c_uint64)]


class Profile(C.Structure):
    _fields_ = [("ms_signature", C.c_double), ("ms_group", C.c_double), ("ms_split", C.c_double),
                ("ms_leaf", C.c_double), ("ms_encode", C.c_double), ("ms_total", C.c_double),
                ("split_nodes", C.c_uint64), ("split_trials", C.c_uint64), ("split_evals", C.c_uint64),
                ("leaf_nodes", C.c_uint64), ("leaf_trials", C.c_uint64), ("leaf_evals", C.c_uint64),
                ("launches", C.c_uint32), ("split_levels", C.c_uint32),
                ("leaf_evals_executed", C.c_uint64), ("split_evals_executed", C.c_uint64)]


class KeySet(C.Structure):
    _fields_ = [("keys", C.c_void_p), ("bytes", C.c_void_p), ("offsets", C.c_void_p), ("n", C.c_uint64),
                ("leaf_size", C.c_uint32), ("bucket_size", C.c_uint32), ("leaf_extra", C.c_uint32),
                ("reserved", C.c_uint32)]


class ServerConfig(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_uint64), ("max_build_batch", C.c_uint32), ("max_lookup_batch", C.c_uint64),
                ("build_workers", C.c_uint32)]


class Completion(C.Structure):
    _fields_ = [("request_id", C.c_uint64), ("structure_id", C.c_uint64), ("items", C.c_uint64),
                ("kind", C.c_int32), ("status", C.c_int32), ("queue_ms", C.c_double), ("latency_ms", C.c_double),
                ("batch_size", C.c_uint32)]


class ServerStats(C.Structure):
    _fields_ = [("resident_structures", C.c_uint64), ("resident_bytes", C.c_uint64), ("in_flight_bytes", C.c_uint64),
                ("queued_builds", C.c_uint64), ("queued_lookups", C.c_uint64), ("keys_built", C.c_uint64),
                ("queries_answered", C.c_uint64)]


class Tuning(C.Structure):
    _fields_ = [("leaf_warps", C.c_uint32), ("leaf_chunk", C.c_uint32), ("leaf_seeds_per_lane", C.c_uint32),
                ("split_warps", C.c_uint32 * 3), ("leaf_two_phase", C.c_uint32)]


def _tuning_dict(t: Tuning) -> dict:
    return {"leaf_warps": t.leaf_warps, "leaf_chunk": t.leaf_chunk, "leaf_seeds_per_lane": t.leaf_seeds_per_lane,
            "split_warps": list(t.split_warps), "leaf_two_phase": t.leaf_two_phase}


class RecSplitError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = _lib
        msg = lib.recsplit_strerror(code).decode() if lib else str(code)
        detail = lib.recsplit_last_error().decode() if lib else ""
        super().__init__(f"{where}: {msg} ({code}){': ' + detail if detail else ''}")
        self.code = code


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise OSError(f"{LIB_PATH} is missing: build it with `python -m paper_1910_06416_gb300.build`")
            L = C.CDLL(LIB_PATH)
            p, u64, u32, i = C.c_void_p, C.c_uint64, C.c_uint32, C.c_int
            L.recsplit_build_u64.argtypes = [p, u64, u32, u32, p, C.POINTER(p)]
            L.recsplit_build.argtypes = [p, u64, u32, u32, p, C.POINTER(p)]
            L.recsplit_build_bytes.argtypes = [p, p, u64, u32, u32, p, C.POINTER(p)]
            L.recsplit_build_perfect_u64.argtypes = [p, u64, u32, u32, u32, p, C.POINTER(p)]
            L.recsplit_build_perfect_bytes.argtypes = [p, p, u64, u32, u32, u32, p, C.POINTER(p)]
            L.recsplit_lookup_u64.argtypes = [p, p, u64, p, p]
            L.recsplit_lookup.argtypes = [p, p, u64, p, p]
            L.recsplit_lookup_bytes.argtypes = [p, p, p, u64, p, p]
            L.recsplit_serialize.argtypes = [p, p, C.c_size_t, C.POINTER(C.c_size_t)]
            L.recsplit_deserialize.argtypes = [p, C.c_size_t, p, C.POINTER(p)]
            L.recsplit_stats.argtypes = [p, C.POINTER(Stats)]
            L.recsplit_free.argtypes = [p]
            L.recsplit_free.restype = None
            L.recsplit_strerror.argtypes = [i]
            L.recsplit_strerror.restype = C.c_char_p
            L.recsplit_last_error.argtypes = []
            L.recsplit_last_error.restype = C.c_char_p
            L.recsplit_golomb_rice_params.argtypes = [u32, u64, p]
            L.recsplit_golomb_rice_params_extra.argtypes = [u32, u32, u64, p]
            L.recsplit_set_profiling.argtypes = [i]
            L.recsplit_last_profile.argtypes = [C.POINTER(Profile)]
            L.recsplit_lookup_u64_static.argtypes = [p, p, u64, p, p]
            L.recsplit_build_batch.argtypes = [p, u32, p, p]
            L.recsplit_get_tuning.argtypes = [u32, p]
            L.recsplit_set_timeout_ms.argtypes = [u32]
            L.recsplit_inject_alloc_failure.argtypes = [C.c_int64]
            L.recsplit_set_tuning.argtypes = [u32, p]
            L.recsplit_autotune.argtypes = [u32, u32, u64, p, p]
            L.recsplit_server_create.argtypes = [p, p]
            L.recsplit_server_destroy.argtypes = [p]
            L.recsplit_server_destroy.restype = None
            L.recsplit_server_submit_build_u64.argtypes = [p, p, u64, u32, u32, p]
            L.recsplit_server_submit_build_bytes.argtypes = [p, p, p, u64, u32, u32, p]
            L.recsplit_server_submit_lookup_u64.argtypes = [p, u64, p, u64, p, p]
            L.recsplit_server_submit_lookup_bytes.argtypes = [p, u64, p, p, u64, p, p]
            L.recsplit_server_poll.argtypes = [p, p, u32, p, i]
            L.recsplit_server_structure.argtypes = [p, u64, p]
            L.recsplit_server_release.argtypes = [p, u64]
            L.recsplit_server_stats.argtypes = [p, p]
            L.recsplit_lookup_batch.argtypes = [p, u32, p, p, u64, p, p]
            L.recsplit_launch_count.argtypes = []
            L.recsplit_launch_count.restype = u64
            for name in ("recsplit_build_u64", "recsplit_build", "recsplit_build_bytes", "recsplit_lookup_u64",
                         "recsplit_lookup", "recsplit_lookup_bytes", "recsplit_serialize", "recsplit_deserialize",
                         "recsplit_stats", "recsplit_golomb_rice_params", "recsplit_set_profiling",
                         "recsplit_last_profile", "recsplit_lookup_u64_static", "recsplit_build_batch",
                         "recsplit_lookup_batch", "recsplit_server_create", "recsplit_server_submit_build_u64",
                         "recsplit_server_submit_build_bytes", "recsplit_server_submit_lookup_u64",
                         "recsplit_server_submit_lookup_bytes", "recsplit_server_poll", "recsplit_server_structure",
                         "recsplit_server_release", "recsplit_server_stats",
                         "recsplit_get_tuning", "recsplit_set_tuning", "recsplit_autotune",
                         "recsplit_set_timeout_ms", "recsplit_inject_alloc_failure"):
                getattr(L, name).restype = i
            _lib = L
    return _lib


def header_functions() -> list[str]:
    """Names of the functions declared in include/recsplit.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(recsplit_[a-z0-9_]+)\s*\(", text)))


def _ptr(x, itemsize=None):
    """Data pointer of a torch tensor or numpy array (None -> NULL).  The
    library reads and writes the elements as one dense array, so a strided
    view, or elements of another size than the argument's (itemsize bytes),
    raise ValueError instead of being misread."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor arguments must be contiguous")
        if itemsize is not None and x.element_size() != itemsize:
            raise ValueError(f"expected {itemsize}-byte elements, got {x.element_size()}-byte {x.dtype}")
        return C.c_void_p(x.data_ptr())
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array arguments must be C-contiguous")
    if itemsize is not None and x.itemsize != itemsize:
        raise ValueError(f"expected {itemsize}-byte elements, got {x.itemsize}-byte {x.dtype}")
    return x.ctypes.data_as(C.c_void_p)


def _u64(x):
    return _ptr(x, 8)


def _u32(x):
    return _ptr(x, 4)


def _u8(x):
    return _ptr(x, 1)


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


def _check(rc: int, where: str):
    if rc != OK:
        raise RecSplitError(rc, where)


def _count(x) -> int:
    return int(x.shape[0])


def _numel(x) -> int:
    return int(x.numel()) if hasattr(x, "numel") else int(x.size)


def _out(out, q: int, name: str = "out"):
    """Pointer of an output array that must hold at least q elements: the
    library writes q results, so a shorter array raises ValueError before the
    call instead of being written past its end."""
    if out is None:
        raise ValueError(f"{name} is required")
    if _numel(out) < q:
        raise ValueError(f"{name} holds {_numel(out)} elements, fewer than the {q} queries")
    return _u64(out)


def _ids(ids, q: int):
    if ids is None or _numel(ids) < q:
        raise ValueError(f"ids must hold at least the {q} structure ids of the queries")
    return _u32(ids)


# ---------------------------------------------------------------- C names
def recsplit_build_u64(keys, leaf_size: int, bucket_size: int, stream=None) -> int:
    """Build from 64-bit keys; returns the opaque handle (an int)."""
    h = C.c_void_p()
    _check(lib().recsplit_build_u64(_u64(keys), _count(keys), leaf_size, bucket_size, _stream(stream), C.byref(h)),
           "recsplit_build_u64")
    return h.value


def recsplit_build(keys, leaf_size: int, bucket_size: int, stream=None) -> int:
    h = C.c_void_p()
    _check(lib().recsplit_build(_u64(keys), _count(keys), leaf_size, bucket_size, _stream(stream), C.byref(h)),
           "recsplit_build")
    return h.value


def recsplit_build_bytes(data, offsets, leaf_size: int, bucket_size: int, stream=None) -> int:
    h = C.c_void_p()
    _check(lib().recsplit_build_bytes(_u8(data), _u64(offsets), _count(offsets) - 1, leaf_size, bucket_size,
                                      _stream(stream), C.byref(h)), "recsplit_build_bytes")
    return h.value


def recsplit_build_perfect_u64(keys, leaf_size: int, bucket_size: int, leaf_extra: int, stream=None) -> int:
    """Perfect, non-minimal variant: leaves of m keys map into m + leaf_extra values."""
    h = C.c_void_p()
    _check(lib().recsplit_build_perfect_u64(_u64(keys), _count(keys), leaf_size, bucket_size, leaf_extra,
                                            _stream(stream), C.byref(h)), "recsplit_build_perfect_u64")
    return h.value


def recsplit_build_perfect_bytes(data, offsets, leaf_size: int, bucket_size: int, leaf_extra: int,
                                 stream=None) -> int:
    h = C.c_void_p()
    _check(lib().recsplit_build_perfect_bytes(_u8(data), _u64(offsets), _count(offsets) - 1, leaf_size,
                                              bucket_size, leaf_extra, _stream(stream), C.byref(h)),
           "recsplit_build_perfect_bytes")
    return h.value


def recsplit_lookup_u64(h: int, keys, out, stream=None) -> None:
    q = _count(keys)
    _check(lib().recsplit_lookup_u64(C.c_void_p(h), _u64(keys), q, _out(out, q), _stream(stream)),
           "recsplit_lookup_u64")


def recsplit_build_batch(sets, stream=None) -> list[int]:
    """Build one structure per set in one pass.  `sets`: sequence of
    (keys, leaf_size, bucket_size) for 64-bit keys or
    (bytes, offsets, leaf_size, bucket_size) for byte strings (device arrays);
    a dict {"leaf_extra": e} as the last element builds that set as the
    perfect, non-minimal variant."""
    arr = (KeySet * max(1, len(sets)))()
    for i, st in enumerate(sets):
        extra = 0
        if st and isinstance(st[-1], dict):
            extra = int(st[-1].get("leaf_extra", 0))
            st = st[:-1]
        if len(st) == 3:
            keys, leaf, b = st
            arr[i] = KeySet(_u64(keys), None, None, _count(keys), leaf, b, extra, 0)
        else:
            data, offs, leaf, b = st
            arr[i] = KeySet(None, _u8(data), _u64(offs), _count(offs) - 1, leaf, b, extra, 0)
    outs = (C.c_void_p * max(1, len(sets)))()
    _check(lib().recsplit_build_batch(C.cast(arr, C.c_void_p), len(sets), _stream(stream), C.cast(outs, C.c_void_p)),
           "recsplit_build_batch")
    return [outs[i] for i in range(len(sets))]


def recsplit_lookup_batch(handles, ids, keys, out, stream=None) -> None:
    """out[i] = lookup of keys[i] in handles[ids[i]]."""
    hs = (C.c_void_p * max(1, len(handles)))(*handles)
    q = _count(keys)
    _check(lib().recsplit_lookup_batch(C.cast(hs, C.c_void_p), len(handles), _ids(ids, q), _u64(keys), q,
                                       _out(out, q), _stream(stream)), "recsplit_lookup_batch")


# ---------------------------------------------------------------- failures
def recsplit_set_timeout_ms(ms: int) -> None:
    _check(lib().recsplit_set_timeout_ms(ms), "recsplit_set_timeout_ms")


def recsplit_inject_alloc_failure(after: int) -> None:
    _check(lib().recsplit_inject_alloc_failure(after), "recsplit_inject_alloc_failure")


# ---------------------------------------------------------------- tuning
def recsplit_get_tuning(leaf_size: int) -> dict:
    t = Tuning()
    _check(lib().recsplit_get_tuning(leaf_size, C.byref(t)), "recsplit_get_tuning")
    return _tuning_dict(t)


def recsplit_set_tuning(leaf_size: int, tuning: dict) -> None:
    t = Tuning(tuning["leaf_warps"], tuning["leaf_chunk"], tuning["leaf_seeds_per_lane"],
               (C.c_uint32 * 3)(*tuning["split_warps"]), tuning.get("leaf_two_phase", 0))
    _check(lib().recsplit_set_tuning(leaf_size, C.byref(t)), "recsplit_set_tuning")


def recsplit_autotune(leaf_size: int, bucket_size: int, sample_keys: int = 1 << 20, stream=None) -> dict:
    t = Tuning()
    _check(lib().recsplit_autotune(leaf_size, bucket_size, sample_keys, _stream(stream), C.byref(t)),
           "recsplit_autotune")
    return _tuning_dict(t)


# ---------------------------------------------------------------- serving
def recsplit_server_create(hbm_budget_bytes=0, max_build_batch=0, max_lookup_batch=0, build_workers=0) -> int:
    cfg = ServerConfig(hbm_budget_bytes, max_build_batch, max_lookup_batch, build_workers)
    h = C.c_void_p()
    _check(lib().recsplit_server_create(C.byref(cfg), C.byref(h)), "recsplit_server_create")
    return h.value


def recsplit_server_destroy(srv: int) -> None:
    lib().recsplit_server_destroy(C.c_void_p(srv))


def recsplit_server_submit_build_u64(srv: int, keys, leaf_size: int, bucket_size: int) -> int:
    rid = C.c_uint64()
    _check(lib().recsplit_server_submit_build_u64(C.c_void_p(srv), _u64(keys), _count(keys), leaf_size, bucket_size,
                                                  C.byref(rid)), "recsplit_server_submit_build_u64")
    return rid.value


def recsplit_server_submit_build_bytes(srv: int, data, offsets, leaf_size: int, bucket_size: int) -> int:
    rid = C.c_uint64()
    _check(lib().recsplit_server_submit_build_bytes(C.c_void_p(srv), _u8(data), _u64(offsets), _count(offsets) - 1,
                                                    leaf_size, bucket_size, C.byref(rid)),
           "recsplit_server_submit_build_bytes")
    return rid.value


def recsplit_server_submit_lookup_u64(srv: int, structure_id: int, keys, out) -> int:
    rid = C.c_uint64()
    q = _count(keys)
    _check(lib().recsplit_server_submit_lookup_u64(C.c_void_p(srv), structure_id, _u64(keys), q, _out(out, q),
                                                   C.byref(rid)), "recsplit_server_submit_lookup_u64")
    return rid.value


def recsplit_server_submit_lookup_bytes(srv: int, structure_id: int, data, offsets, out) -> int:
    rid = C.c_uint64()
    q = _count(offsets) - 1
    _check(lib().recsplit_server_submit_lookup_bytes(C.c_void_p(srv), structure_id, _u8(data), _u64(offsets),
                                                     q, _out(out, q), C.byref(rid)),
           "recsplit_server_submit_lookup_bytes")
    return rid.value


def recsplit_server_poll(srv: int, cap: int = 1024, wait_ms: int = 0) -> list[dict]:
    arr = (Completion * cap)()
    cnt = C.c_uint32()
    _check(lib().recsplit_server_poll(C.c_void_p(srv), C.cast(arr, C.c_void_p), cap, C.byref(cnt), wait_ms),
           "recsplit_server_poll")
    return [{name: getattr(arr[i], name) for name, _ in Completion._fields_} for i in range(cnt.value)]


def recsplit_server_structure(srv: int, structure_id: int) -> int:
    h = C.c_void_p()
    _check(lib().recsplit_server_structure(C.c_void_p(srv), structure_id, C.byref(h)), "recsplit_server_structure")
    return h.value


def recsplit_server_release(srv: int, structure_id: int) -> None:
    _check(lib().recsplit_server_release(C.c_void_p(srv), structure_id), "recsplit_server_release")


def recsplit_server_stats(srv: int) -> dict:
    st = ServerStats()
    _check(lib().recsplit_server_stats(C.c_void_p(srv), C.byref(st)), "recsplit_server_stats")
    return {name: getattr(st, name) for name, _ in ServerStats._fields_}


STATIC_LOOKUP_MAX = 1 << 20


def recsplit_lookup_u64_static(h: int, keys, out, stream=None) -> None:
    """Lookup that allocates no device memory (at most STATIC_LOOKUP_MAX keys)."""
    q = _count(keys)
    _check(lib().recsplit_lookup_u64_static(C.c_void_p(h), _u64(keys), q, _out(out, q), _stream(stream)),
           "recsplit_lookup_u64_static")


def recsplit_lookup(h: int, keys, out, stream=None) -> None:
    q = _count(keys)
    _check(lib().recsplit_lookup(C.c_void_p(h), _u64(keys), q, _out(out, q), _stream(stream)),
           "recsplit_lookup")


def recsplit_lookup_bytes(h: int, data, offsets, out, stream=None) -> None:
    q = _count(offsets) - 1
    _check(lib().recsplit_lookup_bytes(C.c_void_p(h), _u8(data), _u64(offsets), q, _out(out, q),
                                       _stream(stream)), "recsplit_lookup_bytes")


def recsplit_serialize(h: int) -> np.ndarray:
    """The serialized structure as uint64 words."""
    n = C.c_size_t()
    _check(lib().recsplit_serialize(C.c_void_p(h), None, 0, C.byref(n)), "recsplit_serialize")
    buf = np.zeros(n.value // 8, dtype=np.uint64)
    _check(lib().recsplit_serialize(C.c_void_p(h), _ptr(buf), n.value, C.byref(n)), "recsplit_serialize")
    return buf


def recsplit_deserialize(words: np.ndarray, stream=None) -> int:
    words = np.ascontiguousarray(words, dtype=np.uint64)
    h = C.c_void_p()
    _check(lib().recsplit_deserialize(_ptr(words), words.nbytes, _stream(stream), C.byref(h)),
           "recsplit_deserialize")
    return h.value


def recsplit_stats(h: int) -> dict:
    st = Stats()
    _check(lib().recsplit_stats(C.c_void_p(h), C.byref(st)), "recsplit_stats")
    return {name: getattr(st, name) for name, _ in Stats._fields_}


def recsplit_free(h: int) -> None:
    if h:
        lib().recsplit_free(C.c_void_p(h))


def recsplit_strerror(code: int) -> str:
    return lib().recsplit_strerror(code).decode()


def recsplit_last_error() -> str:
    return lib().recsplit_last_error().decode()


def recsplit_golomb_rice_params(leaf_size: int, m_hi: int) -> np.ndarray:
    out = np.zeros(m_hi + 1, dtype=np.uint8)
    _check(lib().recsplit_golomb_rice_params(leaf_size, m_hi, _u8(out)), "recsplit_golomb_rice_params")
    return out


def recsplit_golomb_rice_params_extra(leaf_size: int, leaf_extra: int, m_hi: int) -> np.ndarray:
    out = np.zeros(m_hi + 1, dtype=np.uint8)
    _check(lib().recsplit_golomb_rice_params_extra(leaf_size, leaf_extra, m_hi, _u8(out)),
           "recsplit_golomb_rice_params_extra")
    return out


def recsplit_set_profiling(enabled) -> None:
    """False/0: off; True/1: phase events and work counts; 2: phase events only."""
    _check(lib().recsplit_set_profiling(int(enabled)), "recsplit_set_profiling")


def recsplit_last_profile() -> dict:
    pr = Profile()
    _check(lib().recsplit_last_profile(C.byref(pr)), "recsplit_last_profile")
    return {name: getattr(pr, name) for name, _ in Profile._fields_}


def recsplit_launch_count() -> int:
    return int(lib().recsplit_launch_count())


# ---------------------------------------------------------------- convenience
class Structure:
    """Owning wrapper of a handle (frees it when collected)."""

    def __init__(self, handle: int):
        self.handle = handle

    @classmethod
    def build_u64(cls, keys, leaf_size: int, bucket_size: int, stream=None) -> "Structure":
        return cls(recsplit_build_u64(keys, leaf_size, bucket_size, stream))

    @classmethod
    def build_bytes(cls, data, offsets, leaf_size: int, bucket_size: int, stream=None) -> "Structure":
        return cls(recsplit_build_bytes(data, offsets, leaf_size, bucket_size, stream))

    @classmethod
    def build_perfect_u64(cls, keys, leaf_size: int, bucket_size: int, leaf_extra: int,
                          stream=None) -> "Structure":
        return cls(recsplit_build_perfect_u64(keys, leaf_size, bucket_size, leaf_extra, stream))

    @classmethod
    def build_perfect_bytes(cls, data, offsets, leaf_size: int, bucket_size: int, leaf_extra: int,
                            stream=None) -> "Structure":
        return cls(recsplit_build_perfect_bytes(data, offsets, leaf_size, bucket_size, leaf_extra, stream))

    @classmethod
    def deserialize(cls, words, stream=None) -> "Structure":
        return cls(recsplit_deserialize(words, stream))

    def lookup_u64(self, keys, out, stream=None):
        recsplit_lookup_u64(self.handle, keys, out, stream)
        return out

    def lookup_bytes(self, data, offsets, out, stream=None):
        recsplit_lookup_bytes(self.handle, data, offsets, out, stream)
        return out

    def serialize(self) -> np.ndarray:
        return recsplit_serialize(self.handle)

    def stats(self) -> dict:
        return recsplit_stats(self.handle)

    def free(self):
        if self.handle:
            recsplit_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
