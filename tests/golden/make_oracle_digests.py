"""Writes the stored digests of the workloads in ``digest_cases.py``.

Every structure here is built by the oracle alone (``oracle/``), on the host;
nothing is read from the CUDA library.  Usage:

    python tests/golden/make_oracle_digests.py [--threads N] CASE [CASE ...]

with CASE one of ``leaves``, ``c3``, ``sweep``, ``c4``, ``big``.  Each case
writes ``oracle_digests_<case>.json`` beside this script, recording the
command, the host's core count and the build time.  On 7 cores of a current
x86 host: leaves about 5 minutes, c3 about 30, sweep about 30, c4 about 45,
big about 20 (and about 45 GB of host memory).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

import digest_cases as D  # noqa: E402


def _oracle():
    from oracle import oracle
    oracle.lib()
    return oracle


def _u64_keys(n, seed):
    from paper_1910_06416_gb300 import inputs
    return inputs.u64_keys(n, seed)


def _build_digest(job):
    """(index, full digest, words) of the oracle's structure of one u64 key set."""
    i, n, seed, leaf, bucket = job
    orc = _oracle()
    blob = orc.build_u64(_u64_keys(n, seed), leaf, bucket, threads=1)
    return i, D.words_digest(blob), int(blob.shape[0])


def _pool_digests(jobs, procs):
    """Digests of many independent builds, largest first, in a process pool
    (spawned, so that no state is inherited)."""
    out = {}
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        for i, dig, words in pool.imap_unordered(_build_digest, jobs):
            out[i] = (dig, words)
    return out


def _meta(case, threads, t0):
    return {"case": case, "made_by": "python tests/golden/make_oracle_digests.py --threads "
                                     f"{threads} {case}",
            "host_cores_used": threads, "host": platform.machine(), "seconds": round(time.time() - t0, 1),
            "digest": "sha256 of the serialized structure's 64-bit words, little endian"}


def case_leaves(threads):
    t0 = time.time()
    orc = _oracle()
    rows = []
    for c in D.LARGE_LEAVES:
        blob = orc.build_u64(_u64_keys(c["n"], c["seed"]), c["leaf"], c["bucket"], threads=threads)
        h = orc.header(blob)
        rows.append(dict(c, sha256=D.words_digest(blob), words=int(blob.shape[0]), codes=h["codes"],
                         seeds=orc.decode_bucket(blob, 0)))
        print("leaves", c, rows[-1]["sha256"][:16], flush=True)
    return dict(_meta("leaves", threads, t0), cases=rows)


def case_c3(threads):
    t0 = time.time()
    orc = _oracle()
    c = D.C3
    blob = orc.build_u64(_u64_keys(c["n"], c["seed"]), c["leaf"], c["bucket"], threads=threads)
    h = orc.header(blob)
    buckets = []
    for i in range(h["nbuckets"]):
        s, o = orc.bucket_info(blob, i)
        buckets.append(D.bucket_digest(s, o, orc.decode_bucket(blob, i)))
    return dict(_meta("c3", threads, t0), config=c, sha256=D.words_digest(blob), words=int(blob.shape[0]),
                bits_per_key=orc.bits_per_key(blob), tree_bits=h["tree_bits"], codes=h["codes"],
                bucket_digests=buckets)


def case_sweep(threads):
    t0 = time.time()
    pts = D.sweep_points()
    # the heaviest points (largest leaves) first
    order = sorted(range(len(pts)), key=lambda k: -pts[k][0])
    jobs = [(k, pts[k][2], D.SWEEP_SEED, pts[k][0], pts[k][1]) for k in order]
    res = _pool_digests(jobs, threads)
    rows = [{"leaf": l, "bucket": b, "n": n, "sha256": res[k][0], "words": res[k][1]}
            for k, (l, b, n) in enumerate(pts)]
    return dict(_meta("sweep", threads, t0), seed=D.SWEEP_SEED, points=rows)


def case_c4(threads):
    from paper_1910_06416_gb300 import inputs
    t0 = time.time()
    c = D.C4
    plan = inputs.batch_sets(c["count"], c["lo"], c["hi"], c["seed"])
    # cost grows with the leaf size and the number of keys
    order = sorted(range(len(plan)), key=lambda i: -(plan[i][0] * (50 if plan[i][1] == 12 else 1)))
    jobs = [(i, plan[i][0], plan[i][3], plan[i][1], plan[i][2]) for i in order]
    res = _pool_digests(jobs, threads)
    digests = [res[i][0] for i in range(len(plan))]
    return dict(_meta("c4", threads, t0), config=c, sets=len(plan), keys=int(sum(p[0] for p in plan)),
                sha256_of_all="".join(digests), set_sha256_16=[d[:16] for d in digests],
                set_words=[res[i][1] for i in range(len(plan))])


def case_big(threads):
    from paper_1910_06416_gb300 import inputs
    t0 = time.time()
    c = D.BIG
    keys = np.empty(c["n"], dtype=np.uint64)
    step = 50_000_000
    for a in range(0, c["n"], step):
        b = min(c["n"], a + step)
        keys[a:b] = inputs.splitmix64(c["seed"], b - a, start=a)
    orc = _oracle()
    blob = orc.build_u64(keys, c["leaf"], c["bucket"], threads=threads)
    del keys
    h = orc.header(blob)
    sample = [0, 1, h["nbuckets"] // 2, h["nbuckets"] - 1]
    buckets = {}
    for i in sample:
        s, o = orc.bucket_info(blob, i)
        buckets[str(i)] = D.bucket_digest(s, o, orc.decode_bucket(blob, i))
    return dict(_meta("big", threads, t0), config=c, sha256=D.words_digest(blob), words=int(blob.shape[0]),
                bits_per_key=orc.bits_per_key(blob), bucket_digests=buckets)


CASES = {"leaves": case_leaves, "c3": case_c3, "sweep": case_sweep, "c4": case_c4, "big": case_big}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("cases", nargs="+", choices=sorted(CASES))
    a = ap.parse_args()
    for name in a.cases:
        res = CASES[name](a.threads)
        if name == "c4":
            # the concatenated digests are long: keep one digest of them
            import hashlib
            res["sha256_of_all"] = hashlib.sha256(res["sha256_of_all"].encode()).hexdigest()
        with open(D.path(f"oracle_digests_{name}.json"), "w") as f:
            json.dump(res, f, indent=1)
            f.write("\n")
        print(f"{name}: {res['seconds']} s", flush=True)


if __name__ == "__main__":
    main()
