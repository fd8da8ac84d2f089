"""Benchmark of the flow-analysis hot path on GB300.

Workload (one step): one hour of NetFlow-v5-shaped records, 10,000,000 records in sixty
one-minute windows, against a 5,000-site / 40,000-prefix registry (/8-/30, 20% nested)
with the plain binary-search lookup: per-site sums, rates and flags of all sixty windows
in one persistent launch (a CUDA graph over fixed device buffers).

Prints one JSON line. `value` is records/s of the whole job (all ranks) with the records
resident in HBM; `e2e` is the same metric through the C ABI with host buffers (H2D of
the records and D2H of every window's rates and flags inside the timed region);
`roofline` relates the aggregation kernel's algorithmic bytes to its event-timed
duration; `cpu_baseline` is the CPU oracle on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gnm|reference]
Under torchrun each rank processes its own hour (weak scaling, no collective on the
data path); times are max-reduced over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "flow records/s and % HBM peak (plain vs learned index); p99 window latency"
FALLBACK_HBM_GBS = 6800.0
KERNEL_SOURCES = ["paper_1108_1785_gb300/csrc/agg_kernel.cuh", "paper_1108_1785_gb300/csrc/agg_l2.cu",
                  "paper_1108_1785_gb300/csrc/gnm_internal.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_aggregate_hour_c2_traffic.json")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def workload_desc(n_records, n_windows, reg, n_ranges):
    return (f"hour: {n_records:,} NetFlow-v5-shaped records in {n_windows} one-minute windows; "
            f"{reg.n_sites:,} sites / {reg.n:,} prefixes (/8-/30, 20% nested) -> {n_ranges:,} ranges; "
            f"Zipf(1.0) sites, 85% registered, 30/70 in/out; plain binary search")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("GNM_BENCH_BACKEND", "nccl") == "nccl" else "gloo")
    return world, rank, local


def max_over_ranks(x: float, world: int) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def cpu_oracle_hour(reg, rec, off, n_threads):
    """The CPU oracle over every window of the hour (as it stands); returns seconds."""
    import oracle
    lpm = oracle.LPM(reg.prefix, reg.plen, reg.site)
    t0 = time.perf_counter()
    for w in range(len(off) - 1):
        win = {k: v[off[w]:off[w + 1]] for k, v in rec.items()}
        st, _ = oracle.window(lpm, reg.local_prefix, reg.local_len, reg.n_sites, win, n_threads=n_threads)
        oracle.flags(st, oracle.rates(st), 1e8)
    return time.perf_counter() - t0


def run_reference(args):
    """Reference arm: the CPU oracle on this host's cores, same workload and metric."""
    world, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return 0
    import flowgen as fg
    reg = fg.registry_c2()
    rec, off = fg.hour_records_c2(reg, seed=1)
    n = int(off[-1])
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        cpu_oracle_hour(reg, rec, off, cores)
    ts = [cpu_oracle_hour(reg, rec, off, cores) for _ in range(args.steps)]
    total = sum(ts)
    v = n * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "records/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": workload_desc(n, len(off) - 1, reg, -1).replace(" -> -1 ranges", ""),
                   "parallelism": "host threads"},
        "cpu_baseline": {"value": v, "unit": "records/s", "cores": cores, "kind": "oracle",
                         "sample": f"every step: all {len(off) - 1} windows ({n:,} records), per-length hash "
                                   f"prefix match, {cores} POSIX threads"},
        "e2e": {"value": v, "unit": "records/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gnm", choices=["gnm", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch

    import flowgen as fg
    from paper_1108_1785_gb300 import build, gnm

    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    build.build()
    reg = fg.registry_c2()
    rec, off = fg.hour_records_c2(reg, seed=1 + rank)
    n = int(off[-1])
    n_win = len(off) - 1
    ctx = gnm.Context(device=local, window_slots=2 * n_win + 8)
    ctx.load(reg)
    dev = gnm.Records.to_device(rec)
    ids = np.arange(n_win, dtype=np.uint64)
    # the library's own autotuner picks block size, records per thread, aggregation and
    # registry placement on this workload (outside the timed region)
    tune = ctx.autotune(dev, off, ids)
    info = ctx.registry_info()
    plan = ctx.plan(dev, off, ids)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        plan.launch(stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches = 0
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")  # profilers select the timed steps by this range
        for a, b in ev:
            a.record(stream)
            plan.launch(stream)
            b.record(stream)
            launches += ctx.last_launch_count()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        barrier(world)
    total_ms = ev[0][0].elapsed_time(ev[-1][1])
    kern_ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    total_ms = max_over_ranks(total_ms, world)
    value = n * world * args.steps / (total_ms / 1e3)
    clocks = clk.summary()

    # algorithmic bytes of one launch: 24 B per record read, each window's per-key sums
    # (48 B), rate (8 B) and flag (1 B) written once, the registry read once
    nk = 2 * reg.n_sites
    alg_bytes = 24 * n + n_win * (nk * (48 + 8 + 1) + 4 * 48) + int(info.n_ranges) * 8
    peak, peak_kind = hbm_peak()
    achieved = alg_bytes / (kern_ms / 1e3) / 1e9
    traffic = None
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
        if t.get("kernel_source_hash") == kernel_source_hash() and t.get("records") == n:
            traffic = t["dram_bytes_per_launch"]
    except Exception:
        pass

    out = {
        "metric": METRIC, "value": value, "unit": "records/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": workload_desc(n, n_win, reg, int(info.n_ranges)),
                   "global_batch": n * world, "windows_per_step": n_win * world,
                   "parallelism": f"replicas x{world} (independent hours per GPU)",
                   "lookup": "bsearch, registry " + {gnm.PLACE_SMEM: "in smem", gnm.PLACE_STAGED: "staged (block samples in smem, 64-B blocks in L2)", gnm.PLACE_L2: "in L2"}[info.placement],
                   "l2": "inputs 240 MB per GPU > 129 MB L2; no flush between steps",
                   "launch": "CUDA graph: one persistent aggregation kernel per step (finalise fused)",
                   "tuned": {"block_threads": tune.block_threads, "ctas_per_sm": tune.ctas_per_sm,
                             "unroll": tune.unroll, "aggregation": tune.aggregation, "placement": tune.placement,
                             "default_ms": round(tune.default_ms, 4), "tuned_ms": round(tune.best_ms, 4),
                             "candidates": tune.n_tried}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                     "kernel": "k_aggregate", "kernel_ms": kern_ms, "algorithmic_bytes": alg_bytes},
        "clocks": clocks,
        "gpu_launches": launches,
    }

    if not args.no_e2e:
        # end to end through the C ABI: pinned host records -> library staging -> kernel
        # -> D2H of every window's rates and flags
        pinned = {k: torch.from_numpy(np.ascontiguousarray(rec[k]).view(np.int32)).pin_memory()
                  for k in gnm.FIELDS}
        hostrec = gnm.Records({k: v.numpy() for k, v in pinned.items()})
        rate = np.empty(n_win * nk, np.float64)
        flag = np.empty(n_win * nk, np.uint8)
        e2e_ids = ids + n_win
        for _ in range(max(1, args.warmup)):
            ctx.process_windows(hostrec, off, e2e_ids, stream)
            ctx.windows_results(e2e_ids, rate=rate, flag=flag)
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.process_windows(hostrec, off, e2e_ids, stream)
            ctx.windows_results(e2e_ids, rate=rate, flag=flag)
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, world)
        out["e2e"] = {"value": n * world * args.steps / e2e_s, "unit": "records/s",
                      "h2d_bytes_per_step": 24 * n, "d2h_bytes_per_step": n_win * nk * 9,
                      "api": "gnm_windows_process (host records) + gnm_windows_results"}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        s = cpu_oracle_hour(reg, rec, off, cores)
        out["cpu_baseline"] = {"value": n / s, "unit": "records/s", "cores": cores, "kind": "oracle",
                               "sample": f"the whole step once: {n_win} windows, {n:,} records "
                                         f"({s:.2f} s on {cores} threads)"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    plan.close()
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
