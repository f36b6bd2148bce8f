"""Persistent cache of autotuned launch shapes.

The search launch shapes (warps per node, queue chunk, indices per lane,
leaf test mode) change only the speed of a build, never its result, and the
best ones depend on the GPU model, the leaf size and the bucket size.  This
module keeps the autotuner's choices in a JSON file keyed by those three, so
a process can install a tuned shape without spending the autotuner's sample
builds again.  Host-side bookkeeping only: the tuning itself is
``recsplit_autotune`` in the CUDA library.
"""
import json
import os

from . import recsplit as rs

DEFAULT_PATH = os.path.join(os.path.expanduser("~"), ".cache", "recsplit_gb300_tuning.json")


def cache_key(device_name: str, leaf_size: int, bucket_size: int) -> str:
    return f"{device_name}|l={leaf_size}|b={bucket_size}"


def load(path: str = DEFAULT_PATH) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def save(entries: dict, path: str = DEFAULT_PATH) -> None:
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(entries, f, indent=1, sort_keys=True)
    os.replace(tmp, path)  # readers never see a partial file


def install(device_name: str, leaf_size: int, bucket_size: int, path: str = DEFAULT_PATH) -> dict | None:
    """Installs the cached shape for (device, l, b) with recsplit_set_tuning;
    returns it, or None when the cache has none (or an invalid one)."""
    t = load(path).get(cache_key(device_name, leaf_size, bucket_size))
    if t is None:
        return None
    try:
        rs.recsplit_set_tuning(leaf_size, t)
    except (rs.RecSplitError, KeyError, TypeError):
        return None
    return t


def autotune_cached(device_name: str, leaf_size: int, bucket_size: int, sample_keys: int = 1 << 20,
                    stream=None, path: str = DEFAULT_PATH) -> dict:
    """The cached shape if there is one, else the autotuner's (then cached)."""
    t = install(device_name, leaf_size, bucket_size, path)
    if t is not None:
        return t
    t = rs.recsplit_autotune(leaf_size, bucket_size, sample_keys, stream)
    entries = load(path)
    entries[cache_key(device_name, leaf_size, bucket_size)] = t
    save(entries, path)
    return t
