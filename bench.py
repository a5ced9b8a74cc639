"""Benchmark: split block Bloom filter insert + lookup throughput on GB300.

One step = one pass of the hot path over one batch of the workload: clear the
filter, insert the batch of hashes (appendix add_hash for each), look up the
batch of queries (appendix find_hash for each, packed bitmask out).  The
default workload is the paper's largest size: 100M hashes into a
4,194,304-block (134,217,728 B, HBM-resident) filter in 16M batches, then 1e9
lookups with 10% members.  Inputs are seeded splitmix64 streams generated on
the device before the timed region; the lookup stream (8 GB) is far larger
than L2, so no flush is needed between steps.  The line's ``rows`` add the
other single-filter sizes, each timed the same way: 3e9 hashes at 11
bits/key (4.1 GB) and into 2^30 blocks (32 GiB), each with 1e9 lookups, and
the L2-resident 1 MiB filter with 256M lookups.

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead (a
bounded sample of the same workload on the host cores).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SBBF insert/lookup Gkeys/s"
UNIT = "Gkeys/s"
FALLBACK_HBM_GBS = 6800.0
DOMINANT_KERNEL = "find_kernel"          # single-pass lookups
REGION_KERNEL = "region_find_kernel"     # lookups by region passes
DEFAULT_WORKLOAD = "sbbf_4194304blk_100M_ins_1G_lookup"
# Algorithmic HBM bytes per lookup with an L2-resident filter: the 8-byte
# hash read once plus its 1/8-byte share of the packed result.
LOOKUP_HBM_BYTES_L2_RESIDENT = 8.0 + 1.0 / 8.0
# Measured ceilings of random 32-byte block reads on GB300 (the random-sector
# microbenchmark, paper_2101_01719_gb300/microbench/random_sector.cu):
# blocks resident in L2, and blocks in HBM (where every
# random block costs about 128 bytes of DRAM traffic).
RANDOM_BLOCK_CEILING_L2 = 293.0   # G blocks/s
RANDOM_BLOCK_CEILING_HBM = 40.8   # G blocks/s
# ... and with a filter larger than L2: plus one 32-byte block read.
LOOKUP_HBM_BYTES_HBM_RESIDENT = 8.0 + 32.0 + 1.0 / 8.0
# Insert: the hash, plus a 32-byte block read and written back when the
# filter does not stay in L2.
INSERT_HBM_BYTES_L2_RESIDENT = 8.0
INSERT_HBM_BYTES_HBM_RESIDENT = 8.0 + 32.0 + 32.0


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default=DEFAULT_WORKLOAD)
    p.add_argument("--rows", choices=["auto", "none"], default="auto",
                   help="auto: with the default workload, also time the 11 bits/key, 32 GiB "
                        "and 1 MiB filters as rows of the line")
    p.add_argument("--row-steps", type=int, default=5)
    p.add_argument("--parallelism", choices=["sharded", "replicas"], default="replicas",
                   help="replicas (default): each rank its own copy of the filter and its "
                        "own batch, no data-path collective; sharded: one filter split by "
                        "block range over the ranks, hashes and answers exchanged by "
                        "all-to-all (also runnable with one rank; with N > 1 the default "
                        "line carries it as a row)")
    p.add_argument("--e2e-steps", type=int, default=5)
    p.add_argument("--cpu-seconds", type=float, default=12.0,
                   help="approximate CPU work for the oracle baseline")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--keys", choices=["hashes", "u64", "u32"], default="hashes",
                   help="measurement variant: insert/look up raw 8- or 4-byte keys hashed "
                        "with XXH64 inside the kernels instead of precomputed hashes")
    p.add_argument("--lanes", type=int, choices=[4, 8, 16], default=8,
                   help="measurement variant: 4- or 16-lane blocks (same filter bytes)")
    p.add_argument("--partition", choices=["auto", "on", "off", "regions"], default="auto",
                   help="single-filter workloads: the filter's partitioning mode (auto: the "
                        "library's rule; regions: inserts and lookups by region passes)")
    p.add_argument("--eager", action="store_true",
                   help="launch each kernel from Python instead of replaying CUDA graphs")
    p.add_argument("--requests", type=int, default=0,
                   help="serving workloads: requests per replay (0: the workload's count)")
    p.add_argument("--serial-requests", type=int, default=100_000,
                   help="serving workloads: requests in the serial-launch comparison")
    return p.parse_args(argv)


# ---- distributed plumbing (one process per GPU; units sharded by rank) -----

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_dist(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend)
    return dist if world > 1 else None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value: float, device=None) -> float:
    """Largest value over all ranks (timing only; no data-path collective)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(units_per_rank: list[int], seconds_max: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return sum(units_per_rank) / seconds_max


def step_kernels(f, batches, n_lookup, raw_keys):
    """Kernels one single-filter step launches: the clear, each insert batch
    and the lookup, by region passes, partitioned or not
    (sbbf_region_passes, sbbf_partition_applies; the kernel counts of each
    path are stated in sbbf.h)."""
    hashing = 1 if raw_keys else 0
    n = 1
    for _, cnt in batches:
        ins_passes = f.region_passes(cnt, lookup=False) if not raw_keys else 1
        if ins_passes > 1:
            n += ins_passes
        else:
            n += (3 * ((cnt + 2**34 - 1) // 2**34) + hashing) if f.partition_applies(cnt) else 1
    passes = f.region_passes(n_lookup)  # hashes and fixed-width raw keys alike
    if passes > 1:
        n += passes
    elif f.partition_applies(n_lookup, lookup=True):
        n += 4 * ((n_lookup + 2**31 - 1) // 2**31) + hashing
    else:
        n += 1
    return n


def lookup_slice_start(rank: int, n_lookup: int) -> int:
    """First lookup index of a rank: ranks take disjoint slices of the query
    stream (weak scaling, each rank a replica of the filter)."""
    return rank * n_lookup


# ---- measured peaks, clocks, profile figures --------------------------------

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", self.gpu_id],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def stop(self):
        if self.proc is None:
            return self
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.lines = [l for l in out.splitlines() if l.strip()]
        return self

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() in ("active", "1", "0x1"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# Sources the single-filter lookup kernel (the dominant kernel) is compiled
# from: its template, device helpers, key sources, launch shapes and the
# translation unit that instantiates it.
DOMINANT_SOURCES = ("sbbf_device.cuh", "sbbf_kernels.cuh", "sbbf_keys.cuh", "sbbf_launch.cuh",
                    "sbbf_single.cu")


def kernel_sources_digest() -> str:
    """Digest of the dominant kernel's sources; a stored ncu figure applies
    only while that kernel is unchanged."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2101_01719_gb300", "csrc")
    for name in DOMINANT_SOURCES:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode() + fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str, kernel: str = DOMINANT_KERNEL):
    """DRAM bytes of the dominant kernel per lookup call (all its launches)
    from the committed ncu summary, or None if absent or taken on other
    kernel sources."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    digest = kernel_sources_digest()
    for line in lines:
        parts = line.split()
        if len(parts) >= 4 and parts[0] == workload and parts[1] == kernel:
            if parts[2] == digest:
                return float(parts[3])
    return None


# ---- the workload's config dict (identical in both arms) ----------------------

ROW_WORKLOADS = ("sbbf_128906250blk_3G_ins_1G_lookup", "sbbf_2^30blk_3G_ins_1G_lookup",
                 "sbbf_32768blk_1M_ins_256M_lookup")


def workload_config(w, world: int, lanes: int = 8, keys: str = "hashes") -> dict:
    """What the line measures: the workload, its sizes and the layout of the
    run -- the same dict from our arm and the oracle's, so that the two lines
    compare like for like."""
    return {"workload": w.name, "num_blocks": w.num_blocks * 8 // lanes, "lanes": lanes,
            "keys": ("64-bit hashes" if keys == "hashes"
                     else "%s keys, XXH64 in the kernels" % keys),
            "filter_bytes": w.filter_bytes, "n_insert": w.n_insert,
            "insert_batch": w.insert_batch, "n_lookup": w.n_lookup,
            "member_frac": w.member_frac,
            "l2": "inputs larger than L2 (%.1f GiB lookup stream per step)"
                  % (8 * w.n_lookup / 2**30),
            "parallelism": "independent replicas, lookups sharded by rank"
                           if world > 1 else "single GPU"}


def bytes_per_lookup(w, l2_bytes: int) -> float:
    """Algorithmic HBM bytes per lookup: the hash and its result bit, plus the
    32-byte block when the filter does not stay in L2."""
    l2_resident = w.filter_bytes < l2_bytes / 2
    return LOOKUP_HBM_BYTES_L2_RESIDENT if l2_resident else LOOKUP_HBM_BYTES_HBM_RESIDENT


def bytes_per_insert(w, l2_bytes: int) -> float:
    l2_resident = w.filter_bytes < l2_bytes / 2
    return INSERT_HBM_BYTES_L2_RESIDENT if l2_resident else INSERT_HBM_BYTES_HBM_RESIDENT


def measure_row(name: str, dev, stream, peak: float, l2_bytes: int, steps: int,
                partition_lookups=("auto",)) -> dict:
    """One single-filter workload timed on its own: build the inputs on the
    device, warm up, then time `steps` replays of a CUDA graph of all its
    insert batches (the filter cleared once before; repeated inserts do the
    same work) and of one of its lookup batch with CUDA events on the
    launching stream; the lookup is timed once per partitioning mode listed.
    Members must hit (checked on the last answers)."""
    import torch

    import paper_2101_01719_gb300 as sb
    from paper_2101_01719_gb300 import workloads as wl

    w = wl.WORKLOADS[name]
    f = sb.Filter(w.num_blocks, device=dev)
    ins = wl.gen_inserts(w, 0, w.n_insert, device=dev)
    qry = wl.gen_queries(w, 0, w.n_lookup, device=dev)
    out = torch.empty(sb.out_words(w.n_lookup), dtype=torch.int32, device=dev)
    batches = [(s0, min(w.insert_batch, w.n_insert - s0))
               for s0 in range(0, w.n_insert, w.insert_batch)]

    def insert_all():  # OR is idempotent: a repeated insert does the same work
        for s0, cnt in batches:
            f.insert(ins[s0:s0 + cnt])

    def timed(fn, graph=False):
        """fn's average time over `steps` runs after two warm-up runs; with
        graph, fn is captured once as a CUDA graph and the replays are timed
        (no host launch overhead between the steps)."""
        for _ in range(2):
            fn()
        run = fn
        if graph:
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                fn()
            run = g.replay
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(steps):
            run()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps

    f.clear()
    insert_ms = timed(insert_all, graph=True)
    row = {"filter_bytes": w.filter_bytes, "n_insert": w.n_insert, "n_lookup": w.n_lookup,
           "launch": "CUDA graph of each operation",
           "insert_partitioned": f.partition_applies(batches[0][1]),
           "insert_gkeys_s": round(w.n_insert / (insert_ms / 1e3) / 1e9, 3),
           "insert_ms": round(insert_ms, 4)}
    ib = bytes_per_insert(w, l2_bytes)
    row["insert_roofline"] = {"bytes_per_key": ib,
                              "frac": round(ib * w.n_insert / (insert_ms / 1e3) / 1e9 / peak, 4)}
    lb = bytes_per_lookup(w, l2_bytes)
    row["lookup"] = {}
    modes = {"auto": sb.PARTITION_AUTO, "on": sb.PARTITION_ON, "off": sb.PARTITION_OFF,
             "regions": sb.PARTITION_REGIONS}
    for mode in partition_lookups:
        f.set_partitioning(modes[mode])
        find_ms = timed(lambda: f.find(qry, out=out), graph=True)
        hits = int(sb.count_bits(out, w.n_lookup).item())
        row["lookup"][mode] = {
            "partitioned": f.partition_applies(w.n_lookup, lookup=True),
            "gkeys_s": round(w.n_lookup / (find_ms / 1e3) / 1e9, 3),
            "ms": round(find_ms, 4), "bytes_per_key": lb,
            "roofline_frac": round(lb * w.n_lookup / (find_ms / 1e3) / 1e9 / peak, 4),
            "hit_frac": round(hits / w.n_lookup, 5)}
    f.set_partitioning(sb.PARTITION_AUTO)
    if w.filter_bytes > l2_bytes:  # the verification digest streams every word once
        rb = 1 << 20
        digest_ms = timed(lambda: f.range_digest(rb))
        gbs = w.filter_bytes / (digest_ms / 1e3) / 1e9
        row["digest"] = {"range_blocks": rb, "ms": round(digest_ms, 4), "gbs": round(gbs, 1),
                         "roofline_frac": round(gbs / peak, 4)}
    if l2_bytes < w.filter_bytes <= 8 << 30:
        # union (two reads and one write of every word: 96 B per block) and
        # clear (one write, 32 B per block), streaming
        g = sb.Filter(w.num_blocks, device=dev)
        for name, fn, nbytes in (("union", lambda: f.union_(g), 3 * w.filter_bytes),
                                 ("clear", g.clear, w.filter_bytes)):
            ms = timed(fn)
            gbs = nbytes / (ms / 1e3) / 1e9
            row[name] = {"ms": round(ms, 4), "bytes": nbytes, "gbs": round(gbs, 1),
                         "roofline_frac": round(gbs / peak, 4)}
        del g
    del f, ins, qry, out
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return row


def batched_and_serving_rows(args) -> dict:
    """The batched form (4096 filters, one CUDA-graph launch per step against
    one launch per filter) and the serving form (256 resident filters, a
    1M-request prefix of the 10M-request workload) as rows of the default
    line, with the fields that carry their targets."""
    import copy

    import torch

    a = copy.copy(args)
    a.steps, a.warmup = 3, 1
    a.workload = "sbbf_4096filters_1k-4M_keys_10.5bpk_4x_lookup"
    m = run_multi(a)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    a.workload = "sbbf_serve_256filters_128KiB-1GiB_70pct_lookup"
    a.requests, a.serial_requests = 1_000_000, 50_000
    sv = run_serving(a)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    out = {}
    if m is not None:
        out["batched_4096filters"] = {
            "gkeys_s": m["value"], "ms_per_step": m["ms_per_step"],
            "per_filter_launches_gkeys_s": m["rows"]["per_filter_launches_gkeys_s"],
            "batched_over_per_filter": m["rows"]["batched_over_per_filter"],
            "identical_results": m["rows"]["identical_results"],
            "lookup_roofline_frac": m["roofline"]["frac"], "config": m["config"]["form"]}
    if sv is not None:
        out["serving_256filters_1M_requests"] = {
            "saturation": sv["saturation"], "loads": sv["loads"],
            "serial_per_request_launches": sv["serial_per_request_launches"],
            "batched_same_requests": sv["batched_same_requests"],
            "half_budget": {k: sv["half_budget"][k] for k in
                            ("gkeys_s", "p50_ms", "p99_ms", "budget_bytes")},
            "filter_bytes_total": sv["config"]["filter_bytes_total"]}
    return out


# ---- our arm ----------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch

    import paper_2101_01719_gb300 as sb
    from paper_2101_01719_gb300 import workloads as wl

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = init_dist(world, "nccl")
    w = wl.WORKLOADS[args.workload]
    stream = torch.cuda.current_stream()
    batches = [(s, min(w.insert_batch, w.n_insert - s))
               for s in range(0, w.n_insert, w.insert_batch)]

    # Inputs resident in HBM before timing; each rank takes its own slice of
    # the lookup stream (units sharded by rank, no data-path collective).
    ins = wl.gen_inserts(w, 0, w.n_insert, device=dev)
    qry = wl.gen_queries(w, lookup_slice_start(rank, w.n_lookup), w.n_lookup, device=dev)
    if args.keys == "u32":  # 4-byte keys: the high half of each generated value
        ins = (ins >> 32).to(torch.int32)
        qry = (qry >> 32).to(torch.int32)
    out = torch.empty(sb.out_words(w.n_lookup), dtype=torch.int32, device=dev)
    num_blocks = w.num_blocks * 8 // args.lanes  # the same filter bytes at any lane count
    f = sb.Filter(num_blocks, device=dev, lanes=args.lanes)
    f.set_partitioning({"auto": sb.PARTITION_AUTO, "on": sb.PARTITION_ON,
                        "off": sb.PARTITION_OFF, "regions": sb.PARTITION_REGIONS}[args.partition])
    torch.cuda.synchronize()
    variant = args.keys != "hashes" or args.lanes != 8 or args.partition != "auto"
    do_insert = f.insert if args.keys == "hashes" else f.insert_keys
    do_find = ((lambda q, out: f.find(q, out=out)) if args.keys == "hashes"
               else (lambda q, out: f.find_keys(q, out=out)))

    def insert_all():
        for s0, cnt in batches:
            do_insert(ins[s0:s0 + cnt])

    def step():
        f.clear()
        insert_all()
        do_find(qry, out)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # The step and its parts as CUDA graphs: replays carry no host launch
    # overhead, which otherwise dominates the small workloads.
    graphs = {}
    if not args.eager:
        for name, fn in (("step", step), ("insert", insert_all),
                         ("find", lambda: do_find(qry, out))):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                fn()
            graphs[name] = g
        torch.cuda.synchronize()

    def run_step():
        if graphs:
            graphs["step"].replay()
        else:
            step()

    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", ""))
    gpu_id = uuid if uuid.startswith("GPU-") else ("GPU-" + uuid if uuid else str(local))
    sampler = ClockSampler(gpu_id).start()
    time.sleep(0.3)

    barrier(dist)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        run_step()
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    sampler.stop()
    elapsed_ms = t0.elapsed_time(t1)
    slowest_ms = max_over_ranks(dist, elapsed_ms, dev)

    # Per-kernel durations (same stream as the launches), for the roofline.
    def per_call_ms(fn, reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    reps = max(3, min(args.steps, 50))
    if graphs:
        insert_ms = per_call_ms(graphs["insert"].replay, reps)
        find_ms = per_call_ms(graphs["find"].replay, reps)
    else:
        insert_ms = per_call_ms(insert_all, reps)
        find_ms = per_call_ms(lambda: do_find(qry, out), reps)
    keys_per_step = w.n_insert + w.n_lookup
    value = aggregate([keys_per_step * args.steps] * world, slowest_ms / 1e3) / 1e9

    # correctness spot-check of the timed output (members must hit)
    hits = int(sb.count_bits(out, w.n_lookup).item())

    # end to end through the host-buffer C-ABI calls (pinned host memory)
    e2e = None
    if args.e2e_steps > 0 and not variant:
        h_ins = ins.cpu().pin_memory()
        h_q = qry.cpu().pin_memory()
        h_out = torch.empty(sb.out_words(w.n_lookup), dtype=torch.int32).pin_memory()
        pipe = sb.HostPipe(1 << 24)

        def e2e_run(mode):
            # one call per operation and step: the pipe moves the data itself
            pipe.set_mode(mode)
            h_out.zero_()
            f.clear()
            pipe.insert(f, h_ins)
            pipe.find(f, h_q, h_out)  # warm-up
            barrier(dist)
            torch.cuda.synchronize()
            a = time.perf_counter()
            for _ in range(args.e2e_steps):
                f.clear()
                pipe.insert(f, h_ins)
                pipe.find(f, h_q, h_out)
            torch.cuda.synchronize()
            secs = max_over_ranks(dist, time.perf_counter() - a, dev)
            assert np.array_equal(h_out.numpy(), out.cpu().numpy()), "host path result differs"
            return aggregate([keys_per_step * args.e2e_steps] * world, secs) / 1e9

        # the same calls with the pipe's two ways of moving the data; the line
        # reports the faster and names it
        staged = e2e_run(sb.PIPE_COPY)
        direct = e2e_run(sb.PIPE_DIRECT)
        best = "staged" if staged >= direct else "direct"
        # the host link alone: one pinned host-to-device copy of the lookups
        dq = torch.empty_like(qry)
        dq.copy_(h_q, non_blocking=True)
        torch.cuda.synchronize()
        a = time.perf_counter()
        for _ in range(3):
            dq.copy_(h_q, non_blocking=True)
        torch.cuda.synchronize()
        link_gbs = 3 * h_q.numel() * 8 / (time.perf_counter() - a) / 1e9
        del dq
        e2e = {"value": max(staged, direct), "unit": UNIT,
               "h2d_bytes_per_step": 8 * keys_per_step,
               "d2h_bytes_per_step": 4 * sb.out_words(w.n_lookup),
               "path": "sbbf_insert_hashes_host / sbbf_find_hashes_host on pinned host "
                       "buffers, pipe mode %s" % best,
               "staged_copies": round(staged, 3), "direct_access": round(direct, 3),
               "h2d_link_gbs": round(link_gbs, 1)}
        # host bytes moved per second by the e2e calls, against the link alone
        step_bytes = e2e["h2d_bytes_per_step"] + e2e["d2h_bytes_per_step"]
        e2e["link_frac"] = round(e2e["value"] / keys_per_step * step_bytes / link_gbs, 4)
        del h_ins, h_q, h_out, pipe

    peak, peak_kind = measured_peaks()
    l2_bytes = props.L2_cache_size if hasattr(props, "L2_cache_size") else 126 * 2**20
    l2_resident = w.filter_bytes < l2_bytes / 2
    per_key = bytes_per_lookup(w, l2_bytes)
    key_bytes_less = 4 if args.keys == "u32" else 0  # 4-byte keys instead of 8-byte hashes
    per_key -= key_bytes_less
    achieved = per_key * w.n_lookup / (find_ms / 1e3) / 1e9
    ins_per_key = bytes_per_insert(w, l2_bytes)
    ins_per_key -= key_bytes_less
    ins_achieved = ins_per_key * w.n_insert / (insert_ms / 1e3) / 1e9
    passes = f.region_passes(w.n_lookup)
    lookup_kernel = REGION_KERNEL if passes > 1 else DOMINANT_KERNEL
    traffic = None if variant else profiled_traffic(w.name, lookup_kernel)
    clocks = sampler.summary()
    partitioned = {"insert": f.partition_applies(batches[0][1]),
                   "lookup": f.partition_applies(w.n_lookup, lookup=True)}
    insert_passes = f.region_passes(batches[0][1], lookup=False) if args.keys == "hashes" else 1
    # blocks served from L2: the filter is L2-resident, or each region pass
    # keeps its range of blocks there
    blocks_in_l2 = l2_resident or passes > 1
    step_kernels_n = step_kernels(f, batches, w.n_lookup, args.keys != "hashes")

    rows_extra = {}
    if args.rows == "auto" and not variant and args.workload == DEFAULT_WORKLOAD:
        # free the main workload's device memory (graphs, filter, inputs) first
        graphs.clear()
        do_insert = do_find = None
        del f, ins, qry, out
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        if world == 1:
            for name in ROW_WORKLOADS:
                big = wl.WORKLOADS[name].filter_bytes > (1 << 31)
                rows_extra[name] = measure_row(name, dev, stream, peak, l2_bytes, args.row_steps,
                                               ("auto", "on") if big else ("auto",))
            rows_extra.update(batched_and_serving_rows(args))
        else:  # the same step with one filter sharded over the ranks
            sh = run_sharded(args)
            if sh is not None:
                rows_extra["sharded_over_%d_gpus" % world] = {
                    "gkeys_s": sh["value"], "ms_per_step": sh["ms_per_step"],
                    "num_blocks": sh["config"]["num_blocks"], **sh["rows"],
                    "e2e_gkeys_s": sh["e2e"]["value"]}
    if rank != 0:
        return None
    config = workload_config(w, world, args.lanes, args.keys)
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": round(slowest_ms / args.steps, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded splitmix64 hashes generated on the device)",
        "config": config,
        "path": {"partitioned": partitioned, "insert_region_passes": insert_passes,
                 "lookup_region_passes": passes,
                 "launch": "eager" if args.eager else "CUDA graph of the step"},
        "roofline": {"bound": "hbm", "kernel": lookup_kernel, "launches_per_lookup": passes,
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                     "bytes_per_key": per_key, "traffic": traffic,
                     "insert": {"achieved": round(ins_achieved, 1), "unit": "GB/s",
                                "frac": round(ins_achieved / peak, 4),
                                "bytes_per_key": ins_per_key},
                     # what actually bounds a random-block lookup: one random
                     # 32-byte block per key at the measured random-read rate
                     "random_block_ceiling": {
                         "where": "L2" if blocks_in_l2 else "HBM",
                         "value": (RANDOM_BLOCK_CEILING_L2 if blocks_in_l2
                                   else RANDOM_BLOCK_CEILING_HBM),
                         "unit": "G blocks/s",
                         "frac": round(w.n_lookup / (find_ms / 1e3) / 1e9
                                       / (RANDOM_BLOCK_CEILING_L2 if blocks_in_l2
                                          else RANDOM_BLOCK_CEILING_HBM), 4)}},
        "rows": {"insert_gkeys_s": round(w.n_insert / (insert_ms / 1e3) / 1e9, 3),
                 "lookup_gkeys_s": round(w.n_lookup / (find_ms / 1e3) / 1e9, 3),
                 "insert_ms": round(insert_ms, 5), "lookup_ms": round(find_ms, 5),
                 "lookup_hits": hits, "lookup_hit_frac": round(hits / w.n_lookup, 5),
                 **rows_extra},
        "e2e": e2e,
        "gpu_launches": step_kernels_n * args.steps,
        "clocks": clocks,
    }
    if passes > 1:
        line["roofline"]["note"] = (
            "lookup by %d region passes: achieved counts the method's 40.125 B per lookup "
            "(8 B hash + a 32 B block from HBM + 1/8 B answer) over all passes; the "
            "blocks come from L2 region by region while each pass reads the hashes, so "
            "it can exceed the copy peak" % passes)
    if variant:
        line["roofline"]["note"] = ("variant: e2e, traffic and cpu_baseline are reported "
                                    "for the hash path only")
    if not args.no_cpu_baseline and not variant:
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
    return line



# ---- N ranks: one filter sharded by block range -----------------------------------

def run_sharded(args):
    """Weak scaling of one filter over N GPUs: the filter has N times the
    workload's blocks, each rank owning one workload-sized block range; each
    rank inserts its own n_insert hashes and looks up its own n_lookup
    queries (members drawn from its own inserts), routed to the owners by
    all-to-all exchanges (paper_2101_01719_gb300/sharded.py)."""
    import numpy as np
    import torch

    import paper_2101_01719_gb300 as sb
    from paper_2101_01719_gb300 import workloads as wl
    from paper_2101_01719_gb300.sharded import DeviceOps, ShardedFilter, TorchComm

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = init_dist(world, "nccl")
    import torch.distributed as tdist
    if not tdist.is_initialized():  # one rank: a one-process group, so the exchanges run
        import socket

        with socket.socket() as sock:
            sock.bind(("127.0.0.1", 0))
            port = sock.getsockname()[1]
        tdist.init_process_group("nccl", init_method="tcp://127.0.0.1:%d" % port, rank=0,
                                 world_size=1)
    w = wl.WORKLOADS[args.workload]
    stream = torch.cuda.current_stream()
    num_blocks = w.num_blocks * world
    sf = ShardedFilter(num_blocks, comm=TorchComm(device=dev), ops=DeviceOps(dev))
    ins = wl.gen_inserts(w, rank * w.n_insert, w.n_insert, device=dev)
    qry = torch.empty(w.n_lookup, dtype=torch.int64, device=dev)
    sb.fill_queries(qry, lookup_slice_start(rank, w.n_lookup), wl.seed(w.cfg, wl.ROLE_INSERT),
                    rank * w.n_insert, w.n_insert, wl.seed(w.cfg, wl.ROLE_FRESH),
                    wl.seed(w.cfg, wl.ROLE_MEMBER), wl.member_threshold(w.member_frac))
    batches = [(s0, min(w.insert_batch, w.n_insert - s0))
               for s0 in range(0, w.n_insert, w.insert_batch)]

    def step(ev=None):
        if sf.local is not None:
            sf.local.clear()
        for s0, cnt in batches:
            sf.insert(ins[s0:s0 + cnt])
        if ev is not None:
            ev[0].record(stream)
        out = sf.find(qry)
        if ev is not None:
            ev[1].record(stream)
        return out

    for _ in range(max(args.warmup, 3)):
        out = step()
    torch.cuda.synchronize()
    hits = int(sb.count_bits(out, w.n_lookup).item())
    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", ""))
    sampler = ClockSampler(uuid if uuid.startswith("GPU-") else "GPU-" + uuid).start()
    time.sleep(0.3)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    barrier(dist)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        step(ev[k])
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    sampler.stop()
    slowest_ms = max_over_ranks(dist, t0.elapsed_time(t1), dev)
    find_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
    keys_per_step = w.n_insert + w.n_lookup
    value = aggregate([keys_per_step * args.steps] * world, slowest_ms / 1e3) / 1e9

    # end to end: the step's inputs from pinned host memory, answers back
    h_ins, h_q = ins.cpu().pin_memory(), qry.cpu().pin_memory()
    h_out = torch.empty(sb.out_words(w.n_lookup), dtype=torch.int32).pin_memory()
    barrier(dist)
    torch.cuda.synchronize()
    a = time.perf_counter()
    e2e_steps = max(1, args.e2e_steps)
    for _ in range(e2e_steps):
        ins.copy_(h_ins, non_blocking=True)
        qry.copy_(h_q, non_blocking=True)
        h_out.copy_(step(), non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(dist, time.perf_counter() - a, dev)
    peak, peak_kind = measured_peaks()
    if rank != 0:
        return None
    config = workload_config(w, world)
    config.update({"num_blocks": num_blocks, "filter_bytes": 32 * num_blocks,
                   "n_insert": w.n_insert * world, "n_lookup": w.n_lookup * world,
                   "parallelism": "one filter sharded by block range over %d GPUs "
                                  "(all-to-all of hashes and answer words)" % world})
    return {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": round(slowest_ms / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded splitmix64 hashes generated on the device)",
        "config": config,
        "roofline": {"bound": "hbm", "kernel": "sharded step (route, exchange, shard kernels)",
                     "achieved": round(LOOKUP_HBM_BYTES_HBM_RESIDENT * w.n_lookup
                                       / (find_ms / 1e3) / 1e9, 1),
                     "peak": peak, "unit": "GB/s", "peak_kind": peak_kind,
                     "frac": round(LOOKUP_HBM_BYTES_HBM_RESIDENT * w.n_lookup
                                   / (find_ms / 1e3) / 1e9 / peak, 4),
                     "bytes_per_key": LOOKUP_HBM_BYTES_HBM_RESIDENT, "traffic": None},
        "rows": {"lookup_gkeys_s_per_gpu": round(w.n_lookup / (find_ms / 1e3) / 1e9, 3),
                 "lookup_ms": round(find_ms, 4), "lookup_hit_frac": round(hits / w.n_lookup, 5)},
        "e2e": {"value": round(keys_per_step * e2e_steps * world / e2e_s / 1e9, 3), "unit": UNIT,
                "h2d_bytes_per_step": 8 * keys_per_step,
                "d2h_bytes_per_step": 4 * sb.out_words(w.n_lookup)},
        # per step: the clear; per insert batch the route (count, scan, scatter)
        # and the shard insert; the lookup's route, shard lookup and answer
        # reassembly (NCCL's own kernels not counted)
        "gpu_launches": (1 + 4 * len(batches) + 5) * args.steps,
        "clocks": sampler.summary(),
    }


# ---- many filters: one graph launch per batch vs one launch per filter ---------

def run_multi(args):
    import numpy as np
    import torch

    import paper_2101_01719_gb300 as sb
    from paper_2101_01719_gb300 import workloads as wl

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = init_dist(world, "nccl")
    w = wl.MULTI_WORKLOADS[args.workload]
    stream = torch.cuda.current_stream()
    n_keys, blocks = w.sizes()
    h_ins_off, h_q_off = w.offsets()
    ins, ins_off, q, q_off = wl.gen_multi(w, device=dev)
    n_i, n_q = ins.numel(), q.numel()
    out = torch.empty(sb.out_words(n_q), dtype=torch.int32, device=dev)
    m = sb.MultiFilter(blocks, device=dev)
    m.tune(sb.OP_INSERT, ins, offsets=ins_off)
    m.tune(sb.OP_FIND, q, offsets=q_off)
    tuned = {"insert": m.get_tuning(sb.OP_INSERT, sb.FORM_SEGMENTS),
             "find": m.get_tuning(sb.OP_FIND, sb.FORM_SEGMENTS)}
    keys_per_step = n_i + n_q

    def timed(step_fn, steps, warmup, marks=False):
        for _ in range(warmup):
            step_fn(None)
        torch.cuda.synchronize()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        barrier(dist)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for s_ in range(steps):
            step_fn(ev[s_] if marks else None)
        b.record(stream)
        torch.cuda.synchronize()
        barrier(dist)
        return a.elapsed_time(b), ev

    def graph_step(ev):
        m.clear()
        m.graph_launch(ins, ins_off, q, q_off, out)

    def split_step(ev):
        m.clear()
        if ev:
            ev[0].record(stream)
        m.insert(ins, offsets=ins_off)
        if ev:
            ev[1].record(stream)
        m.find(q, offsets=q_off, out=out)
        if ev:
            ev[2].record(stream)

    def each_step(ev):
        m.clear()
        if ev:
            ev[0].record(stream)
        m.insert_each(ins, h_ins_off)
        if ev:
            ev[1].record(stream)
        m.find_each(q, h_q_off, out=out)
        if ev:
            ev[2].record(stream)

    warm = max(args.warmup, 3)
    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", ""))
    sampler = ClockSampler(uuid if uuid.startswith("GPU-") else "GPU-" + uuid).start()
    time.sleep(0.3)
    graph_ms, _ = timed(graph_step, args.steps, warm)
    sampler.stop()
    graph_out = out.clone()
    split_ms, ev = timed(split_step, args.steps, 1, marks=True)
    each_ms, ev_each = timed(each_step, max(2, min(args.steps, 5)), 1, marks=True)
    each_insert_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in ev_each)
    each_find_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in ev_each)
    same = bool(torch.equal(out, graph_out))
    insert_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
    find_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in ev)
    slowest = max_over_ranks(dist, graph_ms, dev)
    value = aggregate([keys_per_step * args.steps] * world, slowest / 1e3) / 1e9
    each_value = keys_per_step * max(2, min(args.steps, 5)) / (each_ms / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    total_blocks = int(blocks.sum())
    # Algorithmic HBM bytes: every hash once, every filter read once per pass
    # (and written back once by inserts), one result bit per lookup.
    find_bytes = 8.0 * n_q + n_q / 8.0 + 32.0 * total_blocks
    ins_bytes = 8.0 * n_i + 64.0 * total_blocks
    achieved = find_bytes / (find_ms / 1e3) / 1e9
    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": warm, "ms_per_step": round(slowest / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded splitmix64 hashes generated on the device)",
        "config": {"workload": w.name, "n_filters": w.n_filters,
                   "keys_per_filter": [int(n_keys.min()), int(n_keys.max())],
                   "n_insert": n_i, "n_lookup": n_q, "arena_bytes": 32 * total_blocks,
                   "form": "segments, one CUDA graph launch (insert then lookup) per step",
                   "tuning": tuned,
                   "l2": "inputs larger than L2 (%.1f GB per step)" % (8 * keys_per_step / 1e9)},
        "roofline": {"bound": "hbm", "kernel": "find_kernel<Segments>",
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                     "bytes_per_key": round(find_bytes / n_q, 4), "traffic": None,
                     "insert": {"achieved": round(ins_bytes / (insert_ms / 1e3) / 1e9, 1),
                                "frac": round(ins_bytes / (insert_ms / 1e3) / 1e9 / peak, 4),
                                "bytes_per_key": round(ins_bytes / n_i, 4)}},
        "rows": {"insert_gkeys_s": round(n_i / (insert_ms / 1e3) / 1e9, 3),
                 "lookup_gkeys_s": round(n_q / (find_ms / 1e3) / 1e9, 3),
                 "separate_launches_gkeys_s": round(keys_per_step * args.steps
                                                    / (split_ms / 1e3) / 1e9, 3),
                 "per_filter_launches_gkeys_s": round(each_value, 3),
                 "per_filter_insert_gkeys_s": round(n_i / (each_insert_ms / 1e3) / 1e9, 3),
                 "per_filter_lookup_gkeys_s": round(n_q / (each_find_ms / 1e3) / 1e9, 3),
                 "batched_over_per_filter": round(value / each_value, 3),
                 "identical_results": same},
        "gpu_launches": 3 * args.steps,
        "clocks": sampler.summary(),
    }


# ---- serving: continuous batching vs serial per-request launches --------------

def run_serving(args):
    import numpy as np
    import torch

    import paper_2101_01719_gb300 as sb
    from paper_2101_01719_gb300 import workloads as wl

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = wl.SERVING_WORKLOADS[args.workload]
    n_req = args.requests or w.n_requests

    def pct(lat_ns):
        return {"p50_ms": round(float(np.percentile(lat_ns, 50)) / 1e6, 4),
                "p99_ms": round(float(np.percentile(lat_ns, 99)) / 1e6, 4)}

    def make_server(budget):
        srv = sb.Server(budget, max_window_requests=4096, max_inflight_windows=2,
                        max_window_keys=1 << 26, max_pending_requests=1 << 25, device=dev)
        blocks = wl.prefill_server(w, srv, device=dev)
        return srv, blocks

    pool = torch.empty(w.pool_hashes, dtype=torch.int64, device=dev)
    sb.fill_splitmix64(pool, wl.seed(w.cfg, wl.ROLE_FRESH), 0)
    ring_words = 1 << 26
    out = torch.zeros(ring_words + (1 << 16), dtype=torch.int32, device=dev)
    srv, blocks = make_server(w.budget_bytes)
    total_bytes = int(blocks.sum()) * 32

    def replay(server, rate, serial=False, n=n_req):
        op, filt, size, off, arr = w.requests(n, rate)
        rec, _, _ = wl.request_records(op, filt, size, off, pool, out, ring_words)
        a = time.perf_counter()
        lat = server.replay(rec, arr, serial=serial)
        wall = time.perf_counter() - a
        keys = int(size.sum())
        return {"requests": n, "keys": keys, "gkeys_s": round(keys / wall / 1e9, 3),
                "wall_s": round(wall, 3), **pct(lat)}

    warm = replay(srv, float("inf"), n=min(n_req, 20000))
    sat = replay(srv, float("inf"))
    mean_keys = sat["keys"] / sat["requests"]
    cap_req_s = sat["gkeys_s"] * 1e9 / mean_keys
    loads = {}
    for f in (0.5, 0.8, 0.95):
        loads[str(f)] = replay(srv, f * cap_req_s)
    st = srv.stats()
    n_serial = min(n_req, args.serial_requests)
    serial = {"saturation": replay(srv, float("inf"), serial=True, n=n_serial),
              "0.5": replay(srv, 0.5 * cap_req_s, serial=True, n=n_serial)}
    batched_same = {"saturation": replay(srv, float("inf"), n=n_serial),
                    "0.5": replay(srv, 0.5 * cap_req_s, n=n_serial)}
    srv.close()
    srv2, _ = make_server(total_bytes // 2)
    evict = replay(srv2, 0.5 * cap_req_s, n=min(n_req, args.serial_requests))
    evict["budget_bytes"] = total_bytes // 2
    evict["stats"] = srv2.stats()
    srv2.close()
    return {
        "metric": "SBBF serving keys/s; p50/p99 ms", "value": sat["gkeys_s"], "unit": UNIT,
        "n_gpus": 1, "steps": len(loads) + 1, "warmup": 1, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded splitmix64; Poisson arrivals)",
        "config": {"workload": w.name, "n_filters": w.n_filters,
                   "filter_bytes_total": total_bytes, "budget_bytes": w.budget_bytes,
                   "requests": n_req, "lookup_frac": w.lookup_frac,
                   "request_keys": [w.req_lo, w.req_hi], "payload": "device-resident pool",
                   "capacity_req_s": round(cap_req_s, 1)},
        "saturation": sat, "loads": loads, "stats": st,
        "serial_per_request_launches": serial, "batched_same_requests": batched_same,
        "half_budget": evict, "warmup_run": warm,
    }


# ---- the CPU oracle (baseline / reference arm) ---------------------------------

def cpu_baseline(w, seconds: float, steps: int = 1):
    """Time the oracle (scalar C, all host cores) on a bounded sample of the
    workload: the full insert batch, then lookups over a sample of the query
    stream repeated until about `seconds` of CPU time per step."""
    import numpy as np

    import oracle

    cores = oracle.num_cores()
    keys = oracle.splitmix64_fill(0x5BBF000000000000 | (w.cfg << 8), 0, w.n_insert)
    sample = min(w.n_lookup, 1 << 24)
    # the query sample by the same recipe as the device generator
    thr = int(round(w.member_frac * 2.0**32))
    r = oracle.splitmix64_fill(0x5BBF000000000000 | (w.cfg << 8) | 2, 0, sample)
    fresh = oracle.splitmix64_fill(0x5BBF000000000000 | (w.cfg << 8) | 1, 0, sample)
    with np.errstate(over="ignore"):
        idx = ((r & np.uint64(0xFFFFFFFF)) * np.uint64(w.n_insert)) >> np.uint64(32)
    q = np.where((r >> np.uint64(32)) < np.uint64(thr), keys[idx.astype(np.int64)], fresh)
    f = oracle.new_filter(w.num_blocks)
    t_ins = t_find = 0.0
    n_ins = n_find = 0
    used = cores
    for _ in range(steps):
        f[:] = 0
        a = time.perf_counter()
        oracle.insert_mt(f, w.num_blocks, keys, cores)
        t_ins += time.perf_counter() - a
        n_ins += w.n_insert
        a = time.perf_counter()
        _, used = oracle.find_mt(f, w.num_blocks, q[: 1 << 20], cores)
        probe = time.perf_counter() - a
        reps = max(1, int(seconds / steps / max(probe * 16, 1e-6)))
        a = time.perf_counter()
        for _ in range(reps):
            _, used = oracle.find_mt(f, w.num_blocks, q, cores)
        t_find += time.perf_counter() - a
        n_find += reps * sample
    value = (n_ins + n_find) / (t_ins + t_find) / 1e9
    # the oracle as written, on one thread: a 1M-insert / 2M-lookup sample
    g = oracle.new_filter(w.num_blocks)
    ns = min(w.n_insert, 1 << 20)
    a = time.perf_counter()
    oracle.insert(g, w.num_blocks, keys[:ns])
    st_ins = ns / (time.perf_counter() - a) / 1e6
    a = time.perf_counter()
    oracle.find(f, w.num_blocks, q[: 1 << 21])
    st_find = (1 << 21) / (time.perf_counter() - a) / 1e6
    return {"value": round(value, 5), "unit": UNIT, "cores": used, "kind": "oracle",
            "single_thread_insert_mkeys_s": round(st_ins, 2),
            "single_thread_lookup_mkeys_s": round(st_find, 2),
            "sample": "%d inserts + %d lookups (%d x a %d-query prefix of the lookup stream), "
                      "scalar C oracle on %d threads" % (n_ins, n_find, n_find // sample,
                                                          sample, used),
            "insert_mkeys_s": round(n_ins / t_ins / 1e6, 2),
            "lookup_mkeys_s": round(n_find / t_find / 1e6, 2)}


def run_reference(args):
    from paper_2101_01719_gb300 import workloads as wl

    rank, world, _ = dist_env()
    if rank != 0:
        return None  # rank 0 alone runs the CPU oracle
    w = wl.WORKLOADS[args.workload]
    per_step = args.cpu_seconds / max(1, args.steps + args.warmup) * 2
    cpu_baseline(w, per_step, steps=max(args.warmup, 1))  # warm-up
    a = time.perf_counter()
    cb = cpu_baseline(w, per_step, steps=args.steps)
    elapsed = time.perf_counter() - a
    return {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 1),
            "ms_per_step": round(1e3 * elapsed / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (seeded splitmix64 hashes)",
            "config": workload_config(w, world),
            "cpu_baseline": {"value": cb["value"], "unit": UNIT, "cores": cb["cores"],
                             "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main(argv=None):
    args = parse_args(argv)
    from paper_2101_01719_gb300 import workloads as wl
    if args.impl == "reference":
        line = run_reference(args)
    elif args.workload in wl.MULTI_WORKLOADS:
        line = run_multi(args)
    elif args.workload in wl.SERVING_WORKLOADS:
        line = run_serving(args)
    elif args.parallelism == "sharded":
        line = run_sharded(args)
    else:
        line = run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
