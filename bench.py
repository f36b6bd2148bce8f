#!/usr/bin/env python3
"""RecSplit construction + lookup benchmark (one JSON line on rank 0).

Workload (default): 10^7 random byte-string keys of 8..32 bytes (seed 1),
leaf size l = 8, bucket size b = 100, then 10^8 uniform lookups drawn from the
key set.  One step = one build of the whole structure from keys resident in
HBM plus the 10^8 lookups.  `value` is keys built per second (build time),
`lookup` the queries answered per second; `e2e` repeats the build through the
C ABI from pinned host buffers (host->device copy and the read-back of the
structure inside the timed region).

--impl reference times the CPU oracle (the plain C implementation the tests
compare against) on a bounded sample of the same workload.

With torchrun (N > 1) every rank builds its own replica of the workload (the
path has no exchange step on one GPU per box: replicas only); `value` sums
the keys of all ranks over the slowest rank's time.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "build keys/s and lookup Mqueries/s at ℓ=8,b=100 vs INT/HBM roofline; serve p50/p99"
OPS_PER_LEAF_EVAL = 17   # 32-bit instructions of one leaf evaluation (hash, range, one-hot OR)
OPS_PER_SPLIT_EVAL = 20  # 32-bit instructions of one split evaluation (hash, range, part, packed count)
SM_COUNT = 152
LANES_PER_SM_CLK = 128   # 4 sub-partitions x 1 warp instruction (32 lanes) per clock
SM_MAX_MHZ = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=10_000_000)
    ap.add_argument("--queries", type=int, default=100_000_000)
    ap.add_argument("--leaf", type=int, default=8)
    ap.add_argument("--bucket", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="strings", choices=["strings", "u64", "batch", "sweep", "perfect"],
                    help="strings: byte-string keys (default workload); u64: 64-bit keys (seed 0 for leaf 5, "
                         "seed 2 otherwise); batch: 4096 sets of log-uniform sizes with mixed leaf/bucket sizes")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the space-optimal (l=16, b=2000) and batched (4096 sets) entries of the default run")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-workers", type=int, default=0, help="build workers of the serving engine (0: its default)")
    return ap.parse_args()


def max_over_ranks(values, device=None):
    """Element-wise maximum of a list of floats over all ranks (the slowest
    rank's times); the identity outside torch.distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_config(a):
    return {"workload": f"{a.n} random byte-string keys (8-32 B, seed 1), l={a.leaf}, b={a.bucket}, "
                        f"{a.queries} uniform member lookups",
            "n": a.n, "leaf_size": a.leaf, "bucket_size": a.bucket, "queries": a.queries,
            "key_type": "bytes", "l2": "inputs larger than L2 (keys ~280 MB, queries ~2.8 GB)"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        out.update(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=sorted(reasons), samples=len(rows))
        return out


def nvtx_push(name):
    try:
        import torch
        torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def nvtx_pop():
    try:
        import torch
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


# headers every kernel source includes: a change there changes the kernels too
KERNEL_HEADERS = ("device.cuh", "common.h")


def kernel_source_sha(source, root=None):
    """First 16 hex digits of the SHA-256 of a kernel source file followed by
    the shared headers it includes (the hash an ncu summary records)."""
    csrc = os.path.join(root or ROOT, "paper_1910_06416_gb300", "csrc")
    h = hashlib.sha256(open(os.path.join(csrc, source), "rb").read())
    for name in KERNEL_HEADERS:
        path = os.path.join(csrc, name)
        if os.path.exists(path):
            h.update(open(path, "rb").read())
    return h.hexdigest()[:16]


def traffic_from_profiles(kernel_tag, source="search.cu", key="dram_bytes_per_launch"):
    """DRAM bytes recorded by an ncu capture summary (per launch, or with
    key="dram_bytes_all_launches" summed over the captured launches), if the
    kernel source and its shared headers have not changed since (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.md")
    if not os.path.exists(path):
        return None
    sha = kernel_source_sha(source)
    fields = {}
    for line in open(path):
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    if fields.get("source_sha256_16") != sha:
        return None
    try:
        return float(fields[key])
    except (KeyError, ValueError):
        return None


def counters_from_profiles(kernel_tag, source="search.cu"):
    """Issue-slot and DRAM utilisation (percent, first captured launch) from an
    ncu capture summary, if the kernel source has not changed since (else
    None): which of the two limits the kernel."""
    if traffic_from_profiles(kernel_tag, source) is None:
        return None
    want = {"smsp__issue_active.avg.pct_of_peak_sustained_active": "issue_active_pct",
            "gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed": "dram_throughput_pct"}
    out = {}
    for line in open(os.path.join(ROOT, "profiles", f"{kernel_tag}.md")):
        cells = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(cells) >= 3 and cells[0] in want:
            try:
                out[want[cells[0]]] = float(cells[2])
            except ValueError:
                pass
    return out or None


def tuned_shapes(rs, leaf, bucket, sample, stream):
    """Launch shapes for (GPU model, leaf size, bucket size): the persistent
    tuning cache's entry if it has one, else the autotuner's on a seeded
    synthetic sample of `sample` keys (then cached).  Shapes change only the
    speed of a build, never its result."""
    import torch
    from paper_1910_06416_gb300 import tuning_cache
    path = os.environ.get("RECSPLIT_TUNING_CACHE", tuning_cache.DEFAULT_PATH)
    device = torch.cuda.get_device_name()
    hit = tuning_cache.install(device, leaf, bucket, path) is not None
    t = tuning_cache.autotune_cached(device, leaf, bucket, sample, stream, path)
    return dict(t, source="tuning cache" if hit else "autotuned (then cached)")


def timed_repeats(fn, min_s=10.0, max_reps=100000):
    """Runs fn until at least min_s seconds have passed (at most max_reps
    times); returns (repetitions, seconds)."""
    reps, t0 = 0, time.perf_counter()
    while True:
        fn()
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= min_s or reps >= max_reps:
            return reps, dt


def cpu_baseline(a, keys_np):
    """The oracle (plain C, all host cores) on a bounded sample of the
    workload: the first (up to) 10^7 keys, built repeatedly for about 10 s."""
    from oracle import oracle
    from paper_1910_06416_gb300 import inputs
    threads = os.cpu_count() or 1
    ns = min(a.n, 10_000_000)
    sub = inputs.ByteKeys(keys_np.data[:int(keys_np.offsets[ns])], keys_np.offsets[:ns + 1])
    reps, dt = timed_repeats(lambda: oracle.build_bytes(sub.data, sub.offsets, a.leaf, a.bucket, threads=threads))
    # and on one core, on the first 10^6 keys
    n1 = min(a.n, 1_000_000)
    s1 = inputs.ByteKeys(keys_np.data[:int(keys_np.offsets[n1])], keys_np.offsets[:n1 + 1])
    reps1, dt1 = timed_repeats(lambda: oracle.build_bytes(s1.data, s1.offsets, a.leaf, a.bucket, threads=1),
                               min_s=5.0)
    return {"value": ns * reps / dt, "unit": "keys/s", "cores": threads, "kind": "oracle",
            "sample": f"oracle builds of the first {ns} keys of the workload (same l, b; {threads} threads), "
                      f"{reps} builds in {dt:.1f} s",
            "single_core": {"value": n1 * reps1 / dt1, "unit": "keys/s", "cores": 1,
                            "sample": f"{reps1} builds of the first {n1} keys on one thread in {dt1:.1f} s"}}


def serve_run(rs, keys, seconds, rate, leaf, bucket, seed=5, workers=0):
    """Continuous-batching server under Poisson arrivals (mean `rate`/s):
    half builds of log-uniform 10^4..10^7 byte-string keys (slices of the
    key pool), half lookups of log-uniform 10^3..10^6 member queries against
    a resident structure.  Latency is submission to completion."""
    import torch
    rng = np.random.default_rng(seed)
    # request payloads and results in pinned host memory, as a server's
    # receive and reply buffers would be: their copies are then asynchronous
    # DMA instead of the driver's staged copies of pageable memory
    pin_data = torch.from_numpy(keys.data).pin_memory()
    pin_offs = torch.from_numpy(keys.offsets.view(np.int64)).pin_memory()
    data, offsets = pin_data.numpy(), pin_offs.numpy().view(np.uint64)
    ring_cap = 1 << 25
    pin_out = torch.empty(ring_cap, dtype=torch.int64, pin_memory=True)
    ring = pin_out.numpy().view(np.uint64)
    ring_pos = 0
    srv = rs.recsplit_server_create(hbm_budget_bytes=64 << 30, build_workers=workers)
    npool = keys.n
    times, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= seconds:
            break
        times.append(t)
    is_build = rng.random(len(times)) < 0.5
    bsize = np.minimum(np.floor(10 ** rng.uniform(4, 7, len(times))).astype(np.int64), npool)
    qsize = np.floor(10 ** rng.uniform(3, 6, len(times))).astype(np.int64)
    pick = rng.random(len(times))
    resident = []  # (structure id, first key, keys)
    info, live, done = {}, {}, []  # live: lookup id -> its [start, end) of the result ring

    def drain(wait_ms=0):
        for c in rs.recsplit_server_poll(srv, 1024, wait_ms):
            done.append(c)
            kind, start, n = info[c["request_id"]]
            if kind == 0 and c["status"] == 0:
                resident.append((c["structure_id"], start, n))
            live.pop(c["request_id"], None)

    def take(q):
        """q result slots of the ring that no lookup in flight still writes."""
        nonlocal ring_pos
        if ring_pos + q > ring_cap:
            ring_pos = 0
        lo, hi = ring_pos, ring_pos + q
        while any(a < hi and lo < b for a, b in live.values()):
            drain(5)
        ring_pos = hi
        return lo, hi

    t0 = time.perf_counter()
    for i, te in enumerate(times):
        drain()
        delay = t0 + te - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        if not is_build[i] and resident:
            sid, start, n = resident[int(pick[i] * len(resident))]
            q = int(min(qsize[i], n))
            a0 = start + int(rng.integers(0, n - q + 1))
            lo, hi = take(q)
            rid = rs.recsplit_server_submit_lookup_bytes(srv, sid, data, offsets[a0:a0 + q + 1], ring[lo:hi])
            info[rid] = (1, a0, q)
            live[rid] = (lo, hi)
        else:
            n = int(bsize[i])
            start = int(rng.integers(0, npool - n + 1))
            rid = rs.recsplit_server_submit_build_bytes(srv, data, offsets[start:start + n + 1], leaf, bucket)
            info[rid] = (0, start, n)
    while len(done) < len(info):
        drain(50)
    wall = time.perf_counter() - t0
    rs.recsplit_server_destroy(srv)
    res = {"seconds": wall, "rate_hz": rate, "requests": len(done)}
    for kind, name in ((0, "build"), (1, "lookup")):
        ok = [c for c in done if c["kind"] == kind and c["status"] == 0]
        lat = np.array([c["latency_ms"] for c in ok])
        qms = np.array([c["queue_ms"] for c in ok])
        items = sum(c["items"] for c in ok)
        res[name] = {"count": int(lat.size), "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
                     "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
                     "queue_p50_ms": float(np.percentile(qms, 50)) if qms.size else None,
                     "queue_p99_ms": float(np.percentile(qms, 99)) if qms.size else None,
                     "items_per_s": items / wall,
                     "mean_batch": float(np.mean([c["batch_size"] for c in done if c["kind"] == kind] or [0]))}
    failed = [c for c in done if c["status"] != 0]
    res["failed"] = len(failed)
    res["failed_by"] = {}
    for c in failed:
        key = f'{"build" if c["kind"] == 0 else "lookup"} {rs.recsplit_strerror(c["status"])}'
        res["failed_by"][key] = res["failed_by"].get(key, 0) + 1
    return res


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle
    from paper_1910_06416_gb300 import inputs
    threads = os.cpu_count() or 1
    ns = min(a.n, 1_000_000)
    keys = inputs.byte_keys(ns, 1)
    times = []
    for step in range(a.warmup + a.steps):
        t0 = time.perf_counter()
        oracle.build_bytes(keys.data, keys.offsets, a.leaf, a.bucket, threads=threads)
        if step >= a.warmup:
            times.append(time.perf_counter() - t0)
    value = ns * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": dict(workload_config(a), sample_keys=ns),
            "cpu_baseline": {"value": value, "unit": "keys/s", "cores": threads, "kind": "oracle",
                             "sample": f"oracle build of {ns} keys of the workload per step ({threads} threads)"},
            "e2e": {"value": value, "unit": "keys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def add_executed(rooflines, work, leaf_ms, split_ms, peak_ops):
    """Beside the full-model fraction (every trial counted as l or m
    evaluations), the fraction over the evaluations the searches executed:
    the phased leaf tests skip the later parts of most indices, the two-phase
    block test of shared split nodes the last keys of most indices, and every
    round of 32 indices is evaluated whole (counted on the device in the
    work-counting build)."""
    for name, key, ops, ms in (("leaf_search", "leaf_evals_executed", OPS_PER_LEAF_EVAL, leaf_ms),
                               ("split_search", "split_evals_executed", OPS_PER_SPLIT_EVAL, split_ms)):
        if name in rooflines and work.get(key) and ms > 0:
            ach = work[key] * ops / (ms / 1e3) / 1e12
            rooflines[name]["executed"] = {"evals": int(work[key]), "achieved": ach,
                                           "frac": ach / rooflines[name]["peak"],
                                           "evals_per_model_eval": work[key] / max(1, work[name.split("_")[0]
                                                                                          + "_evals"])}


def run_ours(a):
    import torch

    from paper_1910_06416_gb300 import build as lib_build, inputs
    import paper_1910_06416_gb300.recsplit as rs

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        lib_build.build()
    if world > 1:
        torch.distributed.barrier()
    rs.lib()

    keys = inputs.byte_keys(a.n, 1)
    data = torch.from_numpy(keys.data).to(dev)
    offs = torch.from_numpy(keys.offsets.view(np.int64)).to(dev)
    idx = inputs.query_indices(a.n, a.queries, 1)
    qdata, qoffs = inputs.device_byte_queries(keys, idx, device=dev)
    del idx
    qout = torch.empty(a.queries, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)

    # launch shapes of the searches for this leaf size, picked by the autotuner
    # on a seeded synthetic sample (untimed; results do not depend on them)
    tuning = tuned_shapes(rs, a.leaf, a.bucket, a.n, stream.cuda_stream)
    # timed steps record phase events only; the algorithmic work counts come
    # from one more build after the timed region (the searches are
    # deterministic, so every build of this input does the same work)
    rs.recsplit_set_profiling(2)

    def step():
        b0, b1, l1 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        b0.record(stream)
        h = rs.recsplit_build_bytes(data, offs, a.leaf, a.bucket, stream.cuda_stream)
        b1.record(stream)
        rs.recsplit_lookup_bytes(h, qdata, qoffs, qout, stream.cuda_stream)
        l1.record(stream)
        prof = rs.recsplit_last_profile()
        return h, (b0, b1, l1), prof

    for _ in range(a.warmup):
        h, _, _ = step()
        torch.cuda.synchronize()
        rs.recsplit_free(h)

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.4)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = rs.recsplit_launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    records = []
    nvtx_push("timed")  # profilers can restrict a capture to the timed steps
    for _ in range(a.steps):
        h, ev, prof = step()
        records.append((h, ev, prof))
    nvtx_pop()
    t_end.record(stream)
    torch.cuda.synchronize()
    launches = rs.recsplit_launch_count() - launches0
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    stats = rs.recsplit_stats(records[-1][0])
    rs.recsplit_set_profiling(1)
    rs.recsplit_free(rs.recsplit_build_bytes(data, offs, a.leaf, a.bucket, stream.cuda_stream))
    work = rs.recsplit_last_profile()
    rs.recsplit_set_profiling(0)
    for h, _, _ in records:
        rs.recsplit_free(h)

    total_ms = t_start.elapsed_time(t_end)
    build_ms = [ev[0].elapsed_time(ev[1]) for _, ev, _ in records]
    look_ms = [ev[1].elapsed_time(ev[2]) for _, ev, _ in records]
    profs = [p for _, _, p in records]
    total_ms, sb, sl = max_over_ranks([total_ms, sum(build_ms), sum(look_ms)], dev)
    value = world * a.n * a.steps / (sb / 1000.0)
    lookup_qps = world * a.queries * a.steps / (sl / 1000.0)

    # rooflines: searches are integer-issue bound (no tensor cores, no floating
    # point); the lookup reads query strings from HBM and writes indices
    leaf_ms = sum(p["ms_leaf"] for p in profs) / len(profs)
    split_ms = sum(p["ms_split"] for p in profs) / len(profs)
    look_ms_avg = sl / a.steps
    peak_ops = SM_COUNT * LANES_PER_SM_CLK * SM_MAX_MHZ * 1e6
    peak_src = "152 SMs x 128 lanes/clk x 2070 MHz (issue-limited 32-bit integer instructions; derived)"
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    tag = f"strings_n{a.n}_l{a.leaf}_b{a.bucket}"
    lookup_bytes = int(qdata.numel()) + 8 * (a.queries + 1) + 8 * a.queries
    rooflines = {
        "leaf_search": {"bound": "alu", "ms": leaf_ms,
                        "achieved": work["leaf_evals"] * OPS_PER_LEAF_EVAL / (leaf_ms / 1e3) / 1e12,
                        "peak": peak_ops / 1e12, "unit": "Tops/s", "ops_per_eval": OPS_PER_LEAF_EVAL,
                        "peak_source": peak_src, "traffic": traffic_from_profiles(f"leaf_search_{tag}")},
        "split_search": {"bound": "alu", "ms": split_ms,
                         "achieved": work["split_evals"] * OPS_PER_SPLIT_EVAL / (split_ms / 1e3) / 1e12,
                         "peak": peak_ops / 1e12, "unit": "Tops/s", "ops_per_eval": OPS_PER_SPLIT_EVAL,
                         "peak_source": peak_src, "traffic": traffic_from_profiles(f"split_search_{tag}", key="dram_bytes_all_launches")},
        "lookup": {"bound": "hbm", "ms": look_ms_avg, "achieved": lookup_bytes / (look_ms_avg / 1e3) / 1e9,
                   "peak": hbm_peak,
                   "unit": "GB/s", "bytes_per_query": lookup_bytes / a.queries,
                   "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                   "traffic": traffic_from_profiles(f"lookup_{tag}", "lookup.cu")},
    }
    for name, src in (("leaf_search", "search.cu"), ("split_search", "search.cu"), ("lookup", "lookup.cu")):
        rooflines[name]["ncu"] = counters_from_profiles(f"{name}_{tag}" if name != "lookup" else f"lookup_{tag}", src)
    add_executed(rooflines, work, leaf_ms, split_ms, peak_ops)
    for r in rooflines.values():
        r["frac"] = r["achieved"] / r["peak"]
        if r["traffic"] is not None:
            r["traffic"] = r["traffic"] * (a.queries / 1_000_000 if r is rooflines["lookup"] else 1.0)
    kernel = max(rooflines, key=lambda k: rooflines[k]["ms"])
    roofline = dict(rooflines[kernel], kernel=kernel)

    # end to end through the C ABI from pinned host memory
    e2e = None
    if rank == 0:
        hdata = torch.from_numpy(keys.data).pin_memory()
        hoffs = torch.from_numpy(keys.offsets.view(np.int64)).pin_memory()
        ts = []
        blob_bytes = 0
        for k in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = rs.recsplit_build_bytes(hdata, hoffs, a.leaf, a.bucket, stream.cuda_stream)
            blob = rs.recsplit_serialize(h)
            t1 = time.perf_counter()
            rs.recsplit_free(h)
            blob_bytes = blob.nbytes
            ts.append(t1 - t0)
        e2e = {"value": a.n / min(ts), "unit": "keys/s",
               "h2d_bytes_per_step": int(hdata.numel() + 8 * hoffs.numel()), "d2h_bytes_per_step": int(blob_bytes)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": dict(workload_config(a), parallelism=f"replicas{world}", tuning=tuning),
                "lookup": {"value": lookup_qps, "unit": "queries/s"},
                "build_ms": statistics.median(build_ms), "lookup_ms": statistics.median(look_ms),
                "phases_ms": {k: statistics.median(p[k] for p in profs)
                              for k in ("ms_signature", "ms_group", "ms_split", "ms_leaf", "ms_encode", "ms_total")},
                "work": {k: work[k] for k in ("split_nodes", "split_trials", "split_evals", "leaf_nodes",
                                              "leaf_trials", "leaf_evals", "split_evals_executed",
                                              "leaf_evals_executed")},
                "bits_per_key": stats["bits_per_key"], "roofline": roofline, "rooflines": rooflines, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clocks}
        if a.serve_seconds > 0:
            line["serve"] = serve_run(rs, keys, a.serve_seconds, a.serve_rate, a.leaf, a.bucket,
                                      workers=a.serve_workers)
        if not a.no_extras:
            del qdata, qoffs, qout
            torch.cuda.empty_cache()
            line["space_optimal"] = space_optimal_entry(rs, dev, stream)
            torch.cuda.empty_cache()
            line["batched"] = batched_entry(rs, dev, stream)
        if not a.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(a, keys)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def search_rooflines(prof, work, peak_ops):
    peak_src = "152 SMs x 128 lanes/clk x 2070 MHz (issue-limited 32-bit integer instructions; derived)"
    out = {}
    for name, key, ops, ms_key in (("leaf_search", "leaf_evals", OPS_PER_LEAF_EVAL, "ms_leaf"),
                                   ("split_search", "split_evals", OPS_PER_SPLIT_EVAL, "ms_split")):
        ms = prof[ms_key]
        ach = work[key] * ops / (ms / 1e3) / 1e12 if ms > 0 else 0.0
        out[name] = {"bound": "alu", "ms": ms, "achieved": ach, "peak": peak_ops / 1e12, "unit": "Tops/s",
                     "ops_per_eval": ops, "peak_source": peak_src, "frac": ach / (peak_ops / 1e12)}
    add_executed(out, work, prof["ms_leaf"], prof["ms_split"], peak_ops)
    return out


def space_optimal_entry(rs, dev, stream, steps=2, warmup=1, queries=10_000_000):
    """The space-optimal configuration of Table 1: 10^6 64-bit keys (seed 2),
    l = 16, b = 2000 (500 buckets; deep leaf searches of about 8.8e5 trials
    per leaf).  Build keys/s over `steps` builds timed with CUDA events, the
    phase times, the search rooflines (full-model and executed), and member
    lookups/s."""
    import torch
    from paper_1910_06416_gb300 import inputs
    n, leaf, b = 1_000_000, 16, 2000
    keys = torch.from_numpy(inputs.u64_keys(n, 2).view(np.int64)).to(dev)
    q = keys[torch.from_numpy(inputs.query_indices(n, queries, 2)).to(dev)]
    out = torch.empty(queries, dtype=torch.int64, device=dev)
    tuning = tuned_shapes(rs, leaf, b, n, stream.cuda_stream)
    rs.recsplit_set_profiling(2)
    sampler = ClockSampler(dev.index or 0)
    bt, lt, profs = [], [], []
    for step in range(warmup + steps):
        if step == warmup:
            sampler.start()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        h = rs.recsplit_build_u64(keys, leaf, b, stream.cuda_stream)
        e1.record(stream)
        rs.recsplit_lookup_u64(h, q, out, stream.cuda_stream)
        e2.record(stream)
        torch.cuda.synchronize()
        if step >= warmup:
            bt.append(e0.elapsed_time(e1))
            lt.append(e1.elapsed_time(e2))
            profs.append(rs.recsplit_last_profile())
        stats = rs.recsplit_stats(h)
        rs.recsplit_free(h)
    clocks = sampler.stop()
    rs.recsplit_set_profiling(1)
    rs.recsplit_free(rs.recsplit_build_u64(keys, leaf, b, stream.cuda_stream))
    work = rs.recsplit_last_profile()
    rs.recsplit_set_profiling(0)
    prof = {k: statistics.median(p[k] for p in profs)
            for k in ("ms_signature", "ms_group", "ms_split", "ms_leaf", "ms_encode", "ms_total")}
    peak_ops = SM_COUNT * LANES_PER_SM_CLK * SM_MAX_MHZ * 1e6
    build_ms = statistics.median(bt)
    rooflines = search_rooflines(prof, work, peak_ops)
    # DRAM traffic and utilisation of the dominant launches, from their ncu
    # summaries (the full-leaf launch; the two levels on shared nodes)
    tag = f"u64_n{n}_l{leaf}_b{b}"
    for name, summary, key, scope in (
            ("leaf_search", f"leaf_search_{tag}", "dram_bytes_per_launch", "the launch of the full leaves"),
            ("split_search", f"split_shared_{tag}", "dram_bytes_all_launches", "the two levels on shared nodes")):
        rooflines[name]["traffic"] = traffic_from_profiles(summary, key=key)
        rooflines[name]["ncu"] = counters_from_profiles(summary)
        rooflines[name]["traffic_scope"] = scope
    return {"workload": f"{n} 64-bit keys (seed 2), l={leaf}, b={b}, {queries} member lookups",
            "value": n / (build_ms / 1e3), "unit": "keys/s", "build_ms": build_ms, "steps": steps,
            "lookup": {"value": queries / (statistics.median(lt) / 1e3), "unit": "queries/s"},
            "phases_ms": prof, "bits_per_key": stats["bits_per_key"],
            "work": {k: work[k] for k in ("split_nodes", "split_trials", "split_evals", "leaf_nodes", "leaf_trials",
                                          "leaf_evals", "split_evals_executed", "leaf_evals_executed")},
            "rooflines": rooflines, "tuning": tuning, "clocks": clocks}


def batched_entry(rs, dev, stream, steps=2, warmup=1):
    """The batched configuration: 4096 independent structures (sizes
    log-uniform in [10^3, 10^6), seed 3; leaf sizes {5, 8, 12} x bucket sizes
    {5, 100, 2000}) built in one batched pass (timed with CUDA events), against
    one build per launch of the same sets, then 10^9 batched lookups."""
    import torch
    from paper_1910_06416_gb300 import inputs
    plan = inputs.batch_sets(4096, 1000, 1000000, 3)
    keys = [inputs.device_splitmix64(sd, n, device=dev) for n, _, _, sd in plan]
    total = sum(p[0] for p in plan)
    tunings = {}
    for leaf in sorted({p[1] for p in plan}):
        b = max((p for p in plan if p[1] == leaf), key=lambda p: p[0])[2]
        tunings[leaf] = tuned_shapes(rs, leaf, b, 1 << 20, stream.cuda_stream)
    sets = [(k, l, b) for k, (n, l, b, _) in zip(keys, plan)]
    sampler = ClockSampler(dev.index or 0)
    bt, handles, bits = [], None, 0
    for step in range(warmup + steps):
        if step == warmup:
            sampler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hs = rs.recsplit_build_batch(sets, stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if step >= warmup:
            bt.append(e0.elapsed_time(e1))
        if step == warmup + steps - 1:
            handles = hs
            bits = sum(rs.recsplit_stats(h)["total_bits"] for h in hs)
        else:
            for h in hs:
                rs.recsplit_free(h)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    single_bits = 0
    for k, l, b in sets:
        h = rs.recsplit_build_u64(k, l, b, stream.cuda_stream)
        single_bits += rs.recsplit_stats(h)["total_bits"]
        rs.recsplit_free(h)
    e1.record(stream)
    torch.cuda.synchronize()
    single_ms = e0.elapsed_time(e1)
    q, chunk = 1_000_000_000, 100_000_000
    sizes = torch.tensor([p[0] for p in plan], device=dev, dtype=torch.int64)
    flat = torch.cat(keys)
    del keys
    offs = torch.zeros(len(plan) + 1, dtype=torch.int64, device=dev)
    torch.cumsum(sizes, 0, out=offs[1:])
    out = torch.empty(chunk, dtype=torch.int64, device=dev)
    look_ms = 0.0
    for c0 in range(0, q, chunk):
        r = inputs.device_splitmix64(0xC4C4, 2 * chunk, start=2 * c0, device=dev)
        ids = ((r[0::2] >> 1) % len(plan)).to(torch.int32)
        qk = flat[offs[ids.long()] + (r[1::2] >> 1) % sizes[ids.long()]]
        del r
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rs.recsplit_lookup_batch(handles, ids, qk, out, stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        look_ms += e0.elapsed_time(e1)
        del ids, qk
    clocks = sampler.stop()
    for h in handles:
        rs.recsplit_free(h)
    del flat, out
    batch_ms = statistics.median(bt)
    return {"workload": "4096 sets of 64-bit keys, sizes log-uniform in [1e3, 1e6) (seed 3), "
                        "l in {5, 8, 12} x b in {5, 100, 2000}, 1e9 batched lookups",
            "sets": len(plan), "keys": total, "value": total / (batch_ms / 1e3), "unit": "keys/s",
            "batch_ms": batch_ms, "steps": steps,
            "one_per_launch": {"value": total / (single_ms / 1e3), "unit": "keys/s", "ms": single_ms},
            "speedup_vs_one_per_launch": single_ms / batch_ms,
            "bits_per_key": bits / total, "bits_per_key_one_per_launch": single_bits / total,
            "lookup": {"value": q / (look_ms / 1e3), "unit": "queries/s", "queries": q},
            "tuning": {str(k): v for k, v in tunings.items()}, "clocks": clocks}


def run_u64(a):
    """64-bit keys (n, leaf, bucket from the flags): build keys/s and member
    lookups/s, with the same rooflines as the default workload."""
    import torch

    from paper_1910_06416_gb300 import build as lib_build, inputs
    import paper_1910_06416_gb300.recsplit as rs

    lib_build.build()
    rs.lib()
    dev = torch.device("cuda", 0)
    seed = 0 if a.leaf == 5 else 2
    keys_np = inputs.u64_keys(a.n, seed)
    keys = torch.from_numpy(keys_np.view(np.int64)).to(dev)
    qidx = torch.from_numpy(inputs.query_indices(a.n, a.queries, seed)).to(dev)
    queries = keys[qidx]
    del qidx
    out = torch.empty(a.queries, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)
    tuning = tuned_shapes(rs, a.leaf, a.bucket, a.n, stream.cuda_stream)
    rs.recsplit_set_profiling(2)  # phase events only in the timed builds
    bt, lt, profs = [], [], []
    for step in range(a.warmup + a.steps):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        if step == a.warmup:
            nvtx_push("timed")  # profilers can restrict a capture to the timed steps
        e0.record(stream)
        h = rs.recsplit_build_u64(keys, a.leaf, a.bucket, stream.cuda_stream)
        e1.record(stream)
        rs.recsplit_lookup_u64(h, queries, out, stream.cuda_stream)
        e2.record(stream)
        torch.cuda.synchronize()
        if step == a.warmup + a.steps - 1:
            nvtx_pop()
        if step >= a.warmup:
            bt.append(e0.elapsed_time(e1))
            lt.append(e1.elapsed_time(e2))
            profs.append(rs.recsplit_last_profile())
        stats = rs.recsplit_stats(h)
        rs.recsplit_free(h)
    # the work counts (algorithmic and executed) from one more, untimed build
    rs.recsplit_set_profiling(1)
    rs.recsplit_free(rs.recsplit_build_u64(keys, a.leaf, a.bucket, stream.cuda_stream))
    work = rs.recsplit_last_profile()
    rs.recsplit_set_profiling(0)
    prof = {k: statistics.median(p[k] for p in profs)
            for k in ("ms_signature", "ms_group", "ms_split", "ms_leaf", "ms_encode", "ms_total")}
    line = {"metric": "build keys/s (64-bit keys)", "value": a.n / (statistics.median(bt) / 1e3), "unit": "keys/s",
            "workload": "u64", "n": a.n, "leaf_size": a.leaf, "bucket_size": a.bucket, "seed": seed,
            "build_ms": statistics.median(bt), "lookup": {"value": a.queries / (statistics.median(lt) / 1e3),
                                                          "unit": "queries/s", "queries": a.queries},
            "phases_ms": prof,
            "work": {k: work[k] for k in ("split_nodes", "split_trials", "split_evals", "leaf_nodes", "leaf_trials",
                                          "leaf_evals", "split_evals_executed", "leaf_evals_executed")},
            "bits_per_key": stats["bits_per_key"], "tuning": tuning,
            "rooflines": search_rooflines(prof, work, SM_COUNT * LANES_PER_SM_CLK * SM_MAX_MHZ * 1e6)}
    if not a.no_cpu_baseline:
        from oracle import oracle
        threads = os.cpu_count() or 1
        ns = min(a.n, 2_000_000 if a.leaf <= 8 else (20_000 if a.leaf <= 12 else 2_000))
        reps, dt = timed_repeats(lambda: oracle.build_u64(keys_np[:ns], a.leaf, a.bucket, threads=threads))
        line["cpu_baseline"] = {"value": ns * reps / dt, "unit": "keys/s", "cores": threads, "kind": "oracle",
                                "sample": f"oracle builds of the first {ns} keys ({threads} threads), "
                                          f"{reps} builds in {dt:.1f} s"}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(a):
    """4096 independent structures (sizes log-uniform in [10^3, 10^6), seed 3,
    leaf sizes {5, 8, 12} x bucket sizes {5, 100, 2000}) built in one batched
    pass, against one build per launch; then 10^9 batched lookups."""
    import torch

    from paper_1910_06416_gb300 import build as lib_build, inputs
    import paper_1910_06416_gb300.recsplit as rs

    lib_build.build()
    rs.lib()
    dev = torch.device("cuda", 0)
    plan = inputs.batch_sets(4096, 1000, 1000000, 3)
    keys = [inputs.device_splitmix64(sd, n, device=dev) for n, _, _, sd in plan]
    total = sum(p[0] for p in plan)
    stream = torch.cuda.current_stream(dev)
    for leaf in sorted({p[1] for p in plan}):
        b = max((p for p in plan if p[1] == leaf), key=lambda p: p[0])[2]
        rs.recsplit_autotune(leaf, b, 1 << 20, stream.cuda_stream)
    sets = [(k, l, b) for k, (n, l, b, _) in zip(keys, plan)]
    batch_t, bits = [], 0
    for step in range(a.warmup + a.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hs = rs.recsplit_build_batch(sets, stream.cuda_stream)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if step >= a.warmup:
            batch_t.append(dt)
        if step == a.warmup + a.steps - 1:
            bits = sum(rs.recsplit_stats(h)["total_bits"] for h in hs)
            handles = hs
        else:
            for h in hs:
                rs.recsplit_free(h)
    # one build per launch, same sets
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    singles_bits = 0
    for k, l, b in sets:
        h = rs.recsplit_build_u64(k, l, b, stream.cuda_stream)
        singles_bits += rs.recsplit_stats(h)["total_bits"]
        rs.recsplit_free(h)
    torch.cuda.synchronize()
    single_t = time.perf_counter() - t0
    # 10^9 batched lookups (set uniform, then a key uniform in the set)
    q, chunk = 1_000_000_000, 100_000_000
    sizes = torch.tensor([p[0] for p in plan], device=dev, dtype=torch.int64)
    flat = torch.cat(keys)
    offs = torch.zeros(len(plan) + 1, dtype=torch.int64, device=dev)
    torch.cumsum(sizes, 0, out=offs[1:])
    out = torch.empty(chunk, dtype=torch.int64, device=dev)
    look_ms = 0.0
    for c0 in range(0, q, chunk):
        r = inputs.device_splitmix64(0xC4C4, 2 * chunk, start=2 * c0, device=dev)
        ids = ((r[0::2] >> 1) % len(plan)).to(torch.int32)
        qk = flat[offs[ids.long()] + (r[1::2] >> 1) % sizes[ids.long()]]
        del r
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rs.recsplit_lookup_batch(handles, ids, qk, out, stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        look_ms += e0.elapsed_time(e1)
    for h in handles:
        rs.recsplit_free(h)
    line = {"metric": "batched build keys/s vs one build per launch (4096 structures)", "workload": "batch",
            "value": total / statistics.median(batch_t), "unit": "keys/s", "keys": total, "sets": len(plan),
            "batch_s": statistics.median(batch_t), "one_per_launch": {"value": total / single_t, "unit": "keys/s",
                                                                     "seconds": single_t},
            "bits_per_key": bits / total, "bits_per_key_one_per_launch": singles_bits / total,
            "lookup": {"value": q / (look_ms / 1e3), "unit": "queries/s", "queries": q}}
    print(json.dumps(line), flush=True)
    return 0


def model_tree_bits_per_key(rs, leaf, bucket):
    """Expected Golomb-Rice bits per key of the splitting trees (Sec. 5.4):
    a node whose trials succeed with probability p and whose parameter is r
    costs r + 1 / (1 - (1 - p)^(2^r)) bits; p is m!/m^m for a leaf and that
    times k^k/k! per part for a split (Sec. 5.1, 5.2); bucket sizes are
    Poisson(b)."""
    import math
    s_aggr = max(2, -(-(7 * leaf + 10) // 20))
    t_aggr = -(-(21 * leaf + 90) // 100) if leaf >= 7 else 2
    lower, upper = s_aggr * leaf, s_aggr * t_aggr * leaf
    m_hi = int(bucket + 8 * math.sqrt(bucket) + 16)
    r = rs.recsplit_golomb_rice_params(leaf, m_hi)

    def parts(m):
        if m <= leaf:
            return []
        if m > upper:
            left = -(-(m // 2) // upper) * upper
            return [left, m - left]
        unit = leaf if m <= lower else lower
        f = -(-m // unit)
        return [unit] * (f - 1) + [m - unit * (f - 1)]

    memo = {0: 0.0, 1: 0.0}

    def bits(m):
        if m in memo:
            return memo[m]
        ps = parts(m)
        logp = math.lgamma(m + 1) - m * math.log(m)
        for k in ps:
            logp += k * math.log(k) - math.lgamma(k + 1)
        p = math.exp(logp)
        rr = int(r[m])
        v = rr + 1.0 / (-math.expm1((2 ** rr) * math.log1p(-p))) + sum(bits(k) for k in ps)
        memo[m] = v
        return v

    total, w = 0.0, 0.0
    for m in range(0, m_hi + 1):
        pm = math.exp(m * math.log(bucket) - bucket - math.lgamma(m + 1)) if m else math.exp(-bucket)
        total += pm * bits(m)
        w += pm
    return total / w / bucket


def run_sweep(a):
    """Space and construction time over leaf sizes 2..21 and bucket sizes
    {5, 100, 2000} (64-bit keys, seed 4; fewer keys as the leaf searches grow,
    the sizes of the stored oracle digests): the data of the paper's space
    figure and of its construction-time trend (about e per unit of leaf size,
    Sec. 8).  Each point's structure is compared with the oracle's stored
    digest, its bits/key with the Sec. 5.4 model."""
    import hashlib
    import torch

    from paper_1910_06416_gb300 import build as lib_build, inputs
    import paper_1910_06416_gb300.recsplit as rs

    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    import digest_cases as D
    stored = {(p["leaf"], p["bucket"], p["n"]): p["sha256"] for p in (D.load("oracle_digests_sweep.json") or {})
              .get("points", [])}
    lib_build.build()
    rs.lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    rows = []
    keys = {}
    for leaf, b, n in D.sweep_points():
        if n not in keys:
            keys.clear()
            keys[n] = torch.from_numpy(inputs.u64_keys(n, D.SWEEP_SEED).view(np.int64)).to(dev)
        ts = []
        rs.recsplit_set_profiling(2)
        for rep in range(3):
            h = rs.recsplit_build_u64(keys[n], leaf, b, stream.cuda_stream)
            ts.append(rs.recsplit_last_profile()["ms_total"])
            if rep < 2:
                rs.recsplit_free(h)
        st = rs.recsplit_stats(h)
        digest = hashlib.sha256(np.ascontiguousarray(rs.recsplit_serialize(h), dtype="<u8").tobytes()).hexdigest()
        rs.recsplit_free(h)
        rs.recsplit_set_profiling(1)
        rs.recsplit_free(rs.recsplit_build_u64(keys[n], leaf, b, stream.cuda_stream))
        work = rs.recsplit_last_profile()
        rs.recsplit_set_profiling(0)
        want = stored.get((leaf, b, n))
        ms = min(ts[1:])
        rows.append({"leaf": leaf, "bucket": b, "n": n, "bits_per_key": st["bits_per_key"],
                     "tree_bits_per_key": st["tree_bits_per_key"],
                     "model_tree_bits_per_key": model_tree_bits_per_key(rs, leaf, b),
                     "build_ms": ms, "keys_per_s": n / (ms / 1e3),
                     "evals_per_key": (work["leaf_evals"] + work["split_evals"]) / n,
                     "oracle_digest": None if want is None else digest == want})
    for row in rows:
        prev = next((r for r in rows if r["leaf"] == row["leaf"] - 1 and r["bucket"] == row["bucket"]), None)
        if prev:
            row["time_per_key_ratio_to_prev_leaf"] = (row["build_ms"] / row["n"]) / (prev["build_ms"] / prev["n"])
            row["evals_per_key_ratio_to_prev_leaf"] = row["evals_per_key"] / max(prev["evals_per_key"], 1e-30)
    checked = [r["oracle_digest"] for r in rows if r["oracle_digest"] is not None]
    print(json.dumps({"metric": "space and construction time over (leaf, bucket)", "workload": "sweep",
                      "points": len(rows), "oracle_identical": sum(checked), "oracle_checked": len(checked),
                      "rows": rows}), flush=True)
    return 0


def run_perfect(a):
    """Perfect, non-minimal variant: 10^7 64-bit keys (seed 6), l = 8,
    b = 100, leaf range extra e in {0, 1, 2, 4, 8}: build keys/s, bits/key,
    output range per key and 10^8 member lookups/s for each e."""
    import torch

    from paper_1910_06416_gb300 import build as lib_build, inputs
    import paper_1910_06416_gb300.recsplit as rs

    lib_build.build()
    rs.lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    n, q = 10_000_000, 100_000_000
    keys = torch.from_numpy(inputs.u64_keys(n, 6).view(np.int64)).to(dev)
    queries = keys[torch.from_numpy(inputs.query_indices(n, q, 6)).to(dev)]
    out = torch.empty(q, dtype=torch.int64, device=dev)
    rs.recsplit_autotune(8, 100, n, stream.cuda_stream)
    rs.recsplit_set_profiling(2)  # phase events only: the work-counting builds are slower
    rows = []
    for extra in (0, 1, 2, 4, 8):
        bt, lt = [], []
        for rep in range(4):
            h = rs.recsplit_build_perfect_u64(keys, 8, 100, extra, stream.cuda_stream)
            bt.append(rs.recsplit_last_profile()["ms_total"])
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rs.recsplit_lookup_u64(h, queries, out, stream.cuda_stream)
            e1.record(stream)
            torch.cuda.synchronize()
            lt.append(e0.elapsed_time(e1))
            st = rs.recsplit_stats(h)
            rs.recsplit_free(h)
        b_ms, l_ms = statistics.median(bt[1:]), statistics.median(lt[1:])
        rows.append({"leaf_extra": extra, "build_ms": b_ms, "keys_per_s": n / (b_ms / 1e3),
                     "bits_per_key": st["bits_per_key"], "tree_bits_per_key": st["tree_bits_per_key"],
                     "range_per_key": st["range_size"] / n, "lookups_per_s": q / (l_ms / 1e3)})
    print(json.dumps({"metric": "perfect (non-minimal) variant over the leaf range extra", "workload": "perfect",
                      "n": n, "leaf_size": 8, "bucket_size": 100, "queries": q, "rows": rows}), flush=True)
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    if a.workload == "u64":
        return run_u64(a)
    if a.workload == "batch":
        return run_batch(a)
    if a.workload == "perfect":
        return run_perfect(a)
    if a.workload == "sweep":
        return run_sweep(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
