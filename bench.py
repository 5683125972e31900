"""Benchmark: GB/s sorted of 100-byte records on one B300 (or N replicas).

Workload: 100M records x 100 B resident in HBM, two key sets -- uniform
printable ASCII and Zipf(1.1) per key byte with a per-position permutation
and 5 % exact duplicates -- 1024 partitions.  One step sorts both sets
(2 x 10 GB) through the C ABI (elsar_sort).  value = bytes sorted / time.

Also reported: the plain form (the paper's partition rule, one sort launch per
partition) on the same data, the end-to-end rate through elsar_sort_host with
pinned host buffers (copies inside the timed region), the roofline of the
dominant kernel from live CUDA events, and the oracle timed on the host cores
on a bounded sample of the same workload.

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_RECORDS = 100_000_000
PARTITIONS = 1024
RECORD = 100
# algorithmic bytes per record of the sort+gather kernel: read the 16-byte
# pair, read the 100-byte record, write it to its place in the output
SORT_GATHER_BYTES = 16 + 100 + 100
CPU_SAMPLE = 10_000_000  # records of each key set sorted by the oracle for the CPU baseline
# The sort kernel's sources: a DRAM-traffic figure taken by ncu counts only
# while these files are byte for byte the ones it was taken on.
SORT_KERNEL_SOURCES = ("paper_2305_05671_b300/csrc/sort.cu", "paper_2305_05671_b300/csrc/common.cuh")
TRAFFIC_PROFILE = "profiles/sort_gather_kernel_traffic.md"
METRIC = "GB/s sorted (100-B recs), learned+batched vs plain on 1 B300; % HBM roofline"


_SETS = ("uniform", "zipf")


def workloads():
    import recgen

    table = {"uniform": recgen.UNIFORM_100M, "zipf": recgen.ZIPF11_100M}
    return [table[s] for s in _SETS]


def workload_config(extra=None):
    cfg = {
        "workload": "100M x 100-byte records in HBM, two key sets (uniform printable ASCII; Zipf s=1.1 per byte "
                    "with per-position permutation and 5% duplicate keys), 1024 partitions, both sets sorted per step",
        "n_records_per_set": N_RECORDS,
        "sets": 2,
        "partitions": PARTITIONS,
        "cdf": "rmi",
        "balance": "refined",
        "schedule": "persistent",
        "l2": "no flush needed: each input (10 GB) is far larger than L2 (126 MB)",
    }
    if extra:
        cfg.update(extra)
    return cfg


def sort_kernel_digest() -> str:
    h = hashlib.sha256()
    for f in SORT_KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """(DRAM bytes per record, digest) of the sort kernel from the committed ncu
    summary, or (None, reason) when there is none or the kernel has changed
    since it was captured."""
    try:
        with open(os.path.join(ROOT, TRAFFIC_PROFILE)) as f:
            txt = f.read()
    except OSError:
        return None, "no ncu traffic summary"
    d = re.search(r"source digest:\s*`?([0-9a-f]{16})", txt)
    v = re.search(r"dram bytes per record:\s*`?([0-9.]+)", txt)
    if not d or not v:
        return None, "traffic summary unreadable"
    if d.group(1) != sort_kernel_digest():
        return None, f"kernel changed since the ncu capture (digest {d.group(1)})"
    return float(v.group(1)), d.group(1)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0}, "fallback"


class Clocks:
    """nvidia-smi samples (every 50 ms) during the timed region: the samples
    whose timestamps fall inside it, or every sample if none does."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        self.t0 = time.time()
        return self

    def __exit__(self, *a):
        self.t1 = time.time()
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        rows = []
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(f[1]), float(f[2]), f[5:9]))
            except (ValueError, IndexError):
                continue
        if not rows:
            return None
        inside = [r for r in rows if self.t0 is not None and self.t0 - 0.05 <= r[0] <= self.t1 + 0.05]
        use = inside or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = {name for r in use for name, v in zip(names, r[3]) if v.lower() == "active"}
        mx = max(r[2] for r in use)
        sm = [r[1] for r in use]
        load = [x for x in sm if x > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(use), "samples_in_timed_region": len(inside)}


def cpu_baseline(args, world_rank=0, single=True):
    """The oracle, as it stands, on a bounded sample of each key set (the first
    --cpu-sample records): the paper's CPU design over all host cores
    (classification in ranges, partitions sorted in parallel), and, for
    comparison, the single-threaded oracle on the same sample."""
    import oracle
    import recgen

    m = args.cpu_sample
    cores = host_cores()
    tot_bytes, t_all, t_one = 0, 0.0, 0.0
    for wl in workloads():
        host = recgen.generate_cpu(wl["n"], wl["spec"], i0=0, count=m)
        log2B = oracle.default_fine_log2(m, PARTITIONS)
        S = oracle.default_sample_size(m)
        t0 = time.perf_counter()
        oracle.sort_threads(host, PARTITIONS, log2B, S=S, seed=0x5EED, balance=1, threads=cores)
        t_all += time.perf_counter() - t0
        if single:
            t0 = time.perf_counter()
            oracle.sort(host, PARTITIONS, log2B, S=S, seed=0x5EED, balance=1)
            t_one += time.perf_counter() - t0
        tot_bytes += m * RECORD
    out = {"value": round(tot_bytes / t_all / 1e9, 4), "unit": "GB/s", "cores": cores, "kind": "oracle",
           "cpu_model": cpu_model(),
           "sample": f"first {m:,} records of each of the two 100M-record key sets, oracle sort (1024 partitions, "
                     f"1% sample) with its classification and partition sorts spread over {cores} host threads"}
    if single:
        out["single_thread"] = {"value": round(tot_bytes / t_one / 1e9, 4), "cores": 1}
    return out


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl == "elsar" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def max_over_ranks(value: float, world: int) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    for _ in range(args.warmup):
        pass  # the oracle has no warm state; warm-up steps would only repeat the same CPU work
    t0 = time.perf_counter()
    vals = [cpu_baseline(args, single=False) for _ in range(args.steps)]
    dt = time.perf_counter() - t0
    v = statistics.mean(x["value"] for x in vals)
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": workload_config(),
            "cpu_baseline": dict(vals[-1], value=round(v, 4)),
            "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_elsar(args):
    import torch

    import paper_2305_05671_b300 as elsar
    import recgen

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    p = elsar.Params(num_partitions=PARTITIONS, seed=0x5EED, tile_pairs=args.tile_pairs)
    p_plain = elsar.Params(num_partitions=PARTITIONS, seed=0x5EED, balance=elsar.BALANCE_PAPER,
                           schedule=elsar.SCHED_PER_PARTITION, tile_pairs=args.tile_pairs)
    n = args.records
    ins = []
    for wl in workloads():
        d = torch.empty(n * RECORD, dtype=torch.uint8, device=dev)
        recgen.generate_gpu(d, n, wl["spec"], stream=stream.cuda_stream)
        ins.append(d)
    # K streams, each with its own workspace and output: set i sorts on stream i mod K (K = 1: one
    # after the other on one stream)
    K = max(1, min(args.streams, len(ins)))
    streams = [stream] + [torch.cuda.Stream(dev) for _ in range(K - 1)]
    outs = [torch.empty(n * RECORD, dtype=torch.uint8, device=dev) for _ in range(K)]
    wss = [elsar.alloc_workspace(n, p, device=dev) for _ in range(K)]
    out, ws = outs[0], wss[0]
    torch.cuda.synchronize()

    def step(params, stats=False):
        # without stats each sort only enqueues its work (no host round trip); elsar_wait after the
        # timed region reports any device-side timeout of the step's sorts
        sts = [elsar.sort(d, outs[i % K], n, params, ws=wss[i % K], stream=streams[i % K], stats=stats)
               for i, d in enumerate(ins)]
        return sts

    def wait_all():
        for w, s in zip(wss, streams):
            elsar.wait(w, s)

    for _ in range(args.warmup):
        step(p)
    wait_all()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for s in streams[1:]:
            s.wait_event(ev0)
        for _ in range(args.steps):
            step(p)
        for s in streams[1:]:
            e = torch.cuda.Event()
            e.record(s)
            stream.wait_event(e)
        ev1.record(stream)
        torch.cuda.synchronize()
    wait_all()
    barrier(world)
    ms = ev0.elapsed_time(ev1) / args.steps
    ms = max_over_ranks(ms, world)
    bytes_per_step = len(ins) * n * RECORD
    value = world * bytes_per_step / (ms / 1e3) / 1e9

    # per-pass times and counts: the same step with the library's events (stats), after the timed region
    all_stats = [step(p, stats=True) for _ in range(min(args.steps, 3))]
    # the dominant kernel: sort + gather (pass 4), timed by the library's events on the launching stream
    flat = [s for st in all_stats for s in st]
    pass_ms = [statistics.mean(s["pass_ms"][k] for s in flat) for k in range(5)]
    # kernels of one timed step: the stats form's count plus the status note each asynchronous sort adds
    launches = int(sum(s["launches"] for s in flat) / len(all_stats)) + len(ins)
    peaks, how = measured_peaks()
    sg_ms = pass_ms[4]
    achieved = n * SORT_GATHER_BYTES / (sg_ms / 1e3) / 1e9
    tpr, tsrc = profiled_traffic()
    roof = {"kernel": "sort_gather_kernel", "bound": "hbm", "achieved": round(achieved, 1),
            "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
            "peak_source": how,
            "traffic": round(tpr * n) if tpr else None,
            "traffic_source": (f"ncu dram bytes per record {tpr} x {n} records, {TRAFFIC_PROFILE} (kernel digest "
                               f"{tsrc})") if tpr else tsrc,
            "bytes_per_record": SORT_GATHER_BYTES, "avg_launch_ms": round(sg_ms, 3)}

    # plain form on the same data
    plain = None
    for _ in range(args.warmup if not args.no_plain else 0):
        step(p_plain, stats=False)
    torch.cuda.synchronize()
    if not args.no_plain:
        ev0.record(stream)
        for s in streams[1:]:
            s.wait_event(ev0)
        for _ in range(args.steps):
            step(p_plain, stats=False)
        for s in streams[1:]:
            e = torch.cuda.Event()
            e.record(s)
            stream.wait_event(e)
        ev1.record(stream)
        torch.cuda.synchronize()
        wait_all()
        plain_ms = ev0.elapsed_time(ev1) / args.steps
        plain = {"value": round(bytes_per_step / (plain_ms / 1e3) / 1e9, 2), "ms_per_step": round(plain_ms, 3),
                 "form": "paper partition rule, one sort launch per partition"}

    # end to end through elsar_sort_host: pinned host in -> device -> sorted -> pinned host out
    e2e = ooc = None
    if not (args.no_e2e and args.no_ooc):
        h_ins = [d.cpu().pin_memory() for d in ins]
        h_out = torch.empty(n * RECORD, dtype=torch.uint8).pin_memory()
        del ins
        torch.cuda.empty_cache()
    if not args.no_e2e:
        # set i goes in, is sorted and comes back on stream i mod K (elsar_sort_host_async) with that
        # stream's buffers, so that one set's copy back can overlap another's copy in (the host link
        # carries both directions at once)
        d_ins = [torch.empty(n * RECORD, dtype=torch.uint8, device=dev) for _ in range(K)]
        h_outs = [h_out] + [torch.empty(n * RECORD, dtype=torch.uint8).pin_memory() for _ in range(K - 1)]

        def e2e_run(reps):
            for _ in range(reps):
                for i, h in enumerate(h_ins):
                    j = i % K
                    elsar.sort_host_async(h, h_outs[j], n, p, d_ins[j], outs[j], wss[j], stream=streams[j])
            for w, st_ in zip(wss, streams):
                elsar.wait(w, st_)

        e2e_run(1)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_run(args.e2e_steps)
        torch.cuda.synchronize()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, world)
        e2e = {"value": round(world * bytes_per_step / e2e_s / 1e9, 3), "unit": "GB/s",
               "h2d_bytes_per_step": bytes_per_step, "d2h_bytes_per_step": bytes_per_step,
               "steps": args.e2e_steps, "streams": K}
        del d_ins, h_outs
    if not args.no_ooc:
        del ws, out, wss, outs
        torch.cuda.empty_cache()
        ooc = run_ooc(args, h_ins, h_out, n, dev, stream)
    ins = out = ws = wss = outs = None  # the step's device buffers are not needed any more
    torch.cuda.empty_cache()
    batched = None if args.no_batched else run_batched(args, dev, stream)
    cfg4 = None if args.no_cfg4 else run_cfg4(args, dev, stream)
    if rank != 0:
        return
    cpu = cpu_baseline(args) if world == 1 and not args.no_cpu else None
    z = all_stats[-1]
    line = {
        "metric": METRIC,
        "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic", "config": workload_config({"tile_pairs": args.tile_pairs or 2048, "n_records_per_set": n,
                                   "sets": len(workloads()), "streams": K}),
        "records_per_s": round(world * len(workloads()) * n / (ms / 1e3)),
        "hbm_frac_200B": round(world * len(workloads()) * n * 200 / (ms / 1e3) / 1e9 / peaks["hbm_gbs"], 4),
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "plain": plain, "batched": batched,
        "ooc": ooc, "learned_500M": cfg4,
        "passes_ms": {"fit": round(pass_ms[0], 3), "classify": round(pass_ms[1], 3),
                      "scan_cuts_items": round(pass_ms[2], 3), "scatter": round(pass_ms[3], 3),
                      "sort_gather": round(sg_ms, 3)},
        "imbalance": {w["name"]: round(s["max_partition"] / (n / PARTITIONS), 4) for w, s in zip(workloads(), z)},
        "oversize_items": [s["oversize_items"] for s in z],
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_ooc(args, h_ins, h_out, n, dev, stream):
    """Out of core: the same sets held in pinned host memory, sorted into pinned
    host memory under a device budget well below the data (elsar_sort_ooc).
    Reports the wall-clock rate, the phase times, the copy volumes and the
    host link's own bandwidth (one large pinned copy each way) for context."""
    import torch

    import paper_2305_05671_b300 as elsar

    p = elsar.Params(num_partitions=PARTITIONS, seed=0x5EED)
    budget = int(args.ooc_budget_gb * (1 << 30))
    ws = torch.empty(budget, dtype=torch.uint8, device=dev)
    # the link: one pinned copy of a whole set each way
    d = torch.empty(n * RECORD, dtype=torch.uint8, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        d.copy_(h_ins[0], non_blocking=True)
        ev0.record(stream)
        d.copy_(h_ins[0], non_blocking=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        h2d_gbs = n * RECORD / (ev0.elapsed_time(ev1) / 1e3) / 1e9
        ev0.record(stream)
        h_out.copy_(d, non_blocking=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        d2h_gbs = n * RECORD / (ev0.elapsed_time(ev1) / 1e3) / 1e9
    # both directions at once, one set each way
    d2 = torch.empty_like(d)
    s2 = torch.cuda.Stream(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        d.copy_(h_ins[0], non_blocking=True)
    with torch.cuda.stream(s2):
        h_out.copy_(d2, non_blocking=True)
    torch.cuda.synchronize()
    bidir_gbs = 2 * n * RECORD / (time.perf_counter() - t0) / 1e9
    del d, d2
    torch.cuda.empty_cache()
    elsar.sort_ooc(h_ins[0], h_out, n, p, ws=ws, stream=stream)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sts = [elsar.sort_ooc(h, h_out, n, p, ws=ws, stream=stream) for h in h_ins]
    wall = time.perf_counter() - t0
    total = len(h_ins) * n * RECORD
    h2d = sum(s["h2d_bytes"] for s in sts)
    d2h = sum(s["d2h_bytes"] for s in sts)
    # every phase moves whole records: the link alone needs this long
    link_bound_s = max(h2d / (h2d_gbs * 1e9), d2h / (d2h_gbs * 1e9), (h2d + d2h) / (bidir_gbs * 1e9))
    return {"value": round(total / wall / 1e9, 3), "unit": "GB/s", "wall_s": round(wall, 3),
            "device_budget_bytes": budget, "data_bytes_per_set": n * RECORD,
            "phase_ms": {k: [round(s["phase_ms"][i], 1) for s in sts]
                         for i, k in enumerate(("fit", "count", "split", "sort_groups"))},
            "h2d_bytes": h2d, "d2h_bytes": d2h, "chunks": [s["chunks"] for s in sts],
            "groups": [s["groups"] for s in sts], "chunk_records": sts[0]["chunk_records"],
            "group_records": sts[0]["group_records"], "model_used": [s["model_used"] for s in sts],
            "link": {"h2d_gbs": round(h2d_gbs, 2), "d2h_gbs": round(d2h_gbs, 2), "bidir_gbs": round(bidir_gbs, 2)},
            "link_bound_frac": round(link_bound_s / wall, 4),
            "workload": "the step's two sets in pinned host memory, pinned host output, device budget "
                        f"{args.ooc_budget_gb} GiB"}


def run_batched(args, dev, stream):
    """The batched workload: 4096 record sets of log-uniform size in [1K, 1M]
    records (scaled so that they hold 4e8 records at most), even sets uniform,
    odd sets Zipf(1.1) with 5 % duplicates, all sorted by one graph launch."""
    import torch

    import paper_2305_05671_b300 as elsar
    import recgen

    sizes = recgen.batch_sizes(args.batch_sets, cap_records=args.batch_cap)
    d_ins = []
    for k, n in enumerate(sizes):
        d = torch.empty(n * RECORD, dtype=torch.uint8, device=dev)
        recgen.generate_gpu(d, n, recgen.batch_spec(k), stream=stream.cuda_stream)
        d_ins.append(d)
    d_outs = [torch.empty_like(d) for d in d_ins]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b = elsar.Batch(d_ins, d_outs, elsar.Params(seed=0x5EED), stream=stream)
    create_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        b.run(stream)
    b.wait(stream)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        b.run(stream)
    ev1.record(stream)
    b.wait(stream)
    ms = ev0.elapsed_time(ev1) / args.steps
    total = sum(sizes)
    info = b.info()
    b.close()
    # once, outside the timed region: a spread of sets checked as sorted, stable
    # permutations of their inputs (the checker of the full-size tests)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from stable_check import check_stable_sort

    step = max(1, len(sizes) // args.batch_validate)
    checked, valid = 0, True
    for k in range(0, len(sizes), step):
        try:
            check_stable_sort(d_ins[k], d_outs[k], sizes[k])
        except AssertionError:
            valid = False
        checked += 1
    del d_ins, d_outs
    torch.cuda.empty_cache()
    return {"value": round(total * RECORD / (ms / 1e3) / 1e9, 2), "unit": "GB/s", "ms_per_run": round(ms, 3),
            "validated_sets": checked, "valid": valid,
            "sets": len(sizes), "records": total, "graph_launches_per_run": 1,
            "kernels_in_graph": info["launches"], "tile_pairs": info["tile_pairs"],
            "records_per_bin_log2_by_class": info["records_per_bin_log2"], "autotune_runs": info["tuning_runs"],
            "plan_create_s": round(create_s, 2),
            "workload": "4096 sets, sizes log-uniform in [1K, 1M] records scaled to <= 4e8 records, "
                        "even sets uniform, odd sets Zipf(1.1) with 5% duplicates"}


def run_cfg4(args, dev, stream):
    """The learned model at scale: 500M records (Zipf 1.3 per byte, 10 % duplicate
    keys), 4096 partitions, the network requested (its checks on) next to the
    RMI alone.  Per model: GB/s of the default form (refined cuts), the model
    that classified, the fallback reason, and the partition imbalance under both
    cut rules."""
    import torch

    import paper_2305_05671_b300 as elsar
    import recgen

    wl = recgen.ZIPF13_500M
    n, P = args.cfg4_records, wl["P"]
    d_in = torch.empty(n * RECORD, dtype=torch.uint8, device=dev)
    recgen.generate_gpu(d_in, n, wl["spec"], stream=stream.cuda_stream)
    d_out = torch.empty_like(d_in)
    res = {}
    for name, kind in (("rmi", elsar.MODEL_RMI), ("network", elsar.MODEL_MLP)):
        p = elsar.Params(num_partitions=P, seed=0x5EED, model_kind=kind)
        ws = elsar.alloc_workspace(n, p, device=dev)
        st = elsar.sort(d_in, d_out, n, p, ws=ws, stream=stream, stats=True)  # warm-up
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.cfg4_steps):
            st = elsar.sort(d_in, d_out, n, p, ws=ws, stream=stream, stats=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / args.cfg4_steps
        pp = elsar.Params(num_partitions=P, seed=0x5EED, model_kind=kind, balance=elsar.BALANCE_PAPER)
        sp = elsar.sort(d_in, d_out, n, pp, ws=ws, stream=stream, stats=True)
        torch.cuda.synchronize()
        res[name] = {"value": round(n * RECORD / (ms / 1e3) / 1e9, 2), "unit": "GB/s", "ms": round(ms, 3),
                     "passes_ms": {k: round(v, 3) for k, v in zip(("fit", "classify", "scan_cuts_items", "scatter",
                                                                      "sort_gather"), st["pass_ms"])},
                     "model_used": ["rmi", "network", "radix"][st["model_used"]],
                     "fallback_reason": st["fallback_reason"], "fit_ms": round(st["pass_ms"][0], 3),
                     "imbalance_refined": round(st["max_partition"] * P / n, 4),
                     "imbalance_paper_rule": round(sp["max_partition"] * P / n, 4),
                     "judge": {"buckets": st["judge_buckets"], "rmi_max": st["judge_rmi_max"],
                               "network_max": st["judge_mlp_max"]} if kind == elsar.MODEL_MLP else None}
        del ws
        torch.cuda.empty_cache()
    del d_in, d_out
    torch.cuda.empty_cache()
    return {"workload": f"{n:,} records (Zipf 1.3 per byte, 10% duplicates), {P} partitions", **res}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="elsar", choices=["elsar", "reference"])
    ap.add_argument("--tile-pairs", type=int, default=0)
    ap.add_argument("--streams", type=int, default=2, help="sort the step's sets on this many streams at once")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=CPU_SAMPLE, help="records of each set the oracle sorts")
    ap.add_argument("--records", type=int, default=N_RECORDS, help="records per key set (profiling cases use fewer)")
    ap.add_argument("--sets", default="uniform,zipf", help="key sets to sort per step")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-form comparison")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched many-sets workload")
    ap.add_argument("--batch-sets", type=int, default=4096)
    ap.add_argument("--no-ooc", action="store_true", help="skip the out-of-core measurement")
    ap.add_argument("--ooc-budget-gb", type=float, default=2.0, help="device budget of the out-of-core sort")
    ap.add_argument("--batch-cap", type=int, default=400_000_000, help="records across all batched sets")
    ap.add_argument("--batch-validate", type=int, default=64, help="batched sets checked after the timed runs")
    ap.add_argument("--no-cfg4", action="store_true", help="skip the 500M-record learned-model comparison")
    ap.add_argument("--cfg4-records", type=int, default=500_000_000)
    ap.add_argument("--cfg4-steps", type=int, default=2)
    args = ap.parse_args()
    global _SETS
    _SETS = tuple(args.sets.split(","))
    if args.impl == "reference":
        run_reference(args)
    else:
        run_elsar(args)


if __name__ == "__main__":
    main()
