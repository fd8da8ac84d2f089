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
# sources that decide the hour workload's kernels and launch shapes: a DRAM traffic figure
# taken from an ncu capture stands only while these are unchanged
KERNEL_SOURCES = ["paper_1108_1785_gb300/csrc/agg_kernel.cuh", "paper_1108_1785_gb300/csrc/gnm_internal.cuh",
                  "paper_1108_1785_gb300/csrc/agg_radix.cu", "paper_1108_1785_gb300/csrc/agg_keys.cu",
                  "paper_1108_1785_gb300/csrc/kernels_misc.cu", "paper_1108_1785_gb300/csrc/api.cu"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "hour_c2_dram_traffic.json")


def code_only(text: str) -> str:
    """C/CUDA source without comments and whitespace."""
    import re
    code = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    code = re.sub(r"//[^\n]*", "", code)
    return re.sub(r"\s+", "", code)


def kernel_source_hash() -> str:
    """Hash of the kernel sources' code: comments and whitespace do not count."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            h.update(code_only(fh.read()).encode())
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
            f"Zipf(1.0) sites, 85% registered, 30/70 in/out")


LOOKUP_NAMES = {1: "binary search", 2: "learned index (RMI)", 3: "radix directory + binary search"}


def rmi_mode(name):
    """'rmi' = the learned-index workload's model (linear root, 4,096 minimax leaves, leaves
    whose window would exceed 64 split); 'rmi_mse' = the same root with mean-squared-error
    leaves; 'rmi_tE' = 4,096 minimax leaves split above a window of E; 'rmiL' = L minimax
    leaves. Returns (leaves, leaf_fit name, eps_target) or (0, None, 0)."""
    if not name.startswith("rmi"):
        return 0, None, 0
    if name == "rmi_mse":
        return 4096, "mse", 64
    if name.startswith("rmi_t"):
        return 4096, "minimax", int(name[5:])
    return (int(name[3:]) if len(name) > 3 else 4096), "minimax", 64


def learned_vs_plain(gnm, torch, local, steps, warmup, n_records=50_000_000,
                     modes=("bsearch", "radix", "rmi", "rmi_mse", "rmi65536")):
    """Same GPU, same records, 100,000-site / 1,000,000-prefix registry: one window of
    n_records processed with the plain binary search, the radix-directed search and the
    learned index. Results must be bit-exact across the three; throughput per lookup."""
    import flowgen as fg
    reg = fg.registry_c3()
    rec = fg.make_records(reg, n_records, seed=2, p_reg=0.9, zipf_s=0.9)
    dev = gnm.Records.to_device(rec)
    # training keys: 10,000,000 lookups of the plain method (the remote endpoints of other
    # records of the same distribution)
    keys = torch.from_numpy(fg.lookup_keys_c3(reg, 10_000_000).view(np.int32)).cuda()
    peak, peak_kind = hbm_peak()
    stream = torch.cuda.current_stream()
    res, dense, info_out = {}, {}, {}
    for name in modes:
        leaves, fit, target = rmi_mode(name)
        mode = {"bsearch": gnm.LOOKUP_BSEARCH, "radix": gnm.LOOKUP_RADIX}.get(name, gnm.LOOKUP_RMI)
        ctx = gnm.Context(device=local, window_slots=4, lookup_mode=mode)
        ctx.load(reg)
        if leaves:
            rep = ctx.rmi_train(keys, root_kind=gnm.ROOT_LINEAR, n_leaves=leaves, leaf_iters=4,
                                leaf_fit=gnm.FIT_MSE if fit == "mse" else gnm.FIT_MINIMAX, eps_target=target)
            info_out[name] = {"leaves": leaves, "root": "linear", "leaf_fit": fit, "eps_target": target,
                              "models": int(rep.n_models),
                              "split_leaves": int(rep.split_leaves), "eps_max": int(rep.eps_max),
                              "err_max": int(rep.err_max), "eps_mean": round(float(rep.eps_mean), 2),
                              "train_ms": round(float(rep.train_ms), 1), "sweep_ms": round(float(rep.sweep_ms), 1),
                              "train_keys": int(keys.numel())}
            ctx.rmi_violations(reset=True)
        plan = ctx.plan(dev, [0, n_records], [1], kernel_times=True)
        for _ in range(warmup):
            plan.launch(stream)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed")
        a.record(stream)
        for _ in range(steps):
            plan.launch(stream)
        b.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        ms = a.elapsed_time(b) / steps
        per = []
        for _ in range(3):  # per-kernel split of a launch
            plan.launch(stream)
            per.append(plan.kernel_times())
        kms = {nm: round(float(np.mean([q[i][1] for q in per])), 4) for i, (nm, _) in enumerate(per[0])}
        info = ctx.registry_info()
        alg = 24 * n_records + (2 * reg.n_sites * (48 + 8 + 1) + 4 * 48) + int(info.n_ranges) * 8
        gbs = alg / (ms / 1e3) / 1e9
        res[name] = {"records_per_s": n_records / (ms / 1e3), "ms": ms, "achieved_gbs": gbs,
                     "frac": gbs / peak, "launches": ctx.last_launch_count(), "kernels_ms": kms,
                     "lookup": LOOKUP_NAMES.get(int(info.lookup_mode), str(int(info.lookup_mode)))}
        if leaves:
            res[name]["violations"] = ctx.rmi_violations()
            res[name]["model"] = info_out[name]
        dense[name] = ctx.dense(1)
        info_out["n_ranges"] = int(info.n_ranges)
        plan.close()
        ctx.close()
    ref = next(iter(dense))
    exact = all(np.array_equal(dense[k][i], dense[ref][i], equal_nan=(i == 2)) for k in dense for i in range(4))
    return {"workload": f"one window of {n_records:,} records; {reg.n_sites:,} sites / {reg.n:,} prefixes "
                        f"(/16-/30, 30% nested) -> {info_out['n_ranges']:,} ranges; Zipf(0.9), 90% registered",
            "peak_gbs": peak, "peak_kind": peak_kind, "bitexact_across_lookups": bool(exact),
            **res,
            "rmi_speedup_vs_bsearch": (res["bsearch"]["ms"] / res["rmi"]["ms"]
                                       if "bsearch" in res and "rmi" in res else None),
            "best_rmi_speedup_vs_bsearch": (max((res["bsearch"]["ms"] / v["ms"], k) for k, v in res.items()
                                                if k.startswith("rmi"))
                                            if "bsearch" in res and any(k.startswith("rmi") for k in res)
                                            else None)}


def paper_lookup(gnm, torch, local, steps, warmup):
    """The paper's GPU Site Catalog (every registered network expanded into /24 subnets in
    a hash table) against this library's lookups, on the hour's workload shape with the
    prefix lengths such a catalog can hold (/8-/24): same GPU, same records, each shape
    autotuned, results bit-exact across the three."""
    import flowgen as fg
    reg = fg.registry_c2_24()
    rec, off = fg.hour_records_c2(reg, seed=1)
    n, n_win = int(off[-1]), len(off) - 1
    dev = gnm.Records.to_device(rec)
    ids = np.arange(n_win, dtype=np.uint64)
    stream = torch.cuda.current_stream()
    res, dense = {}, {}
    for name, mode in (("hash24", gnm.LOOKUP_HASH24), ("bsearch", gnm.LOOKUP_BSEARCH), ("radix", gnm.LOOKUP_RADIX)):
        ctx = gnm.Context(device=local, window_slots=n_win + 8, lookup_mode=mode)
        ctx.load(reg)
        ctx.autotune(dev, off, ids)
        plan = ctx.plan(dev, off, ids, kernel_times=True)
        for _ in range(warmup):
            plan.launch(stream)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            plan.launch(stream)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        plan.launch(stream)
        res[name] = {"records_per_s": n / (ms / 1e3), "ms": ms,
                     "kernels_ms": {k: round(v, 4) for k, v in plan.kernel_times()}}
        dense[name] = [ctx.dense(int(w)) for w in (0, 29, 59)]
        plan.close()
        ctx.close()
    exact = all(np.array_equal(x, y, equal_nan=True) for k in dense for a_, b_ in zip(dense[k], dense["hash24"])
                for x, y in zip(a_, b_))
    return {"workload": f"hour: {n:,} records in {n_win} windows; {reg.n_sites:,} sites / {reg.n:,} prefixes "
                        "/8-/24 (20% nested) -> a /24 subnet table of "
                        f"{int((np.int64(1) << (24 - reg.plen.astype(np.int64))).sum()):,} subnets",
            "bitexact_across_lookups": bool(exact), **res,
            "hash24_vs_best": min(res["bsearch"]["ms"], res["radix"]["ms"]) / res["hash24"]["ms"]}


def window_c1(gnm, torch, local, reps=1000):
    """One window of 100,000 records against the 500-site registry: per-window latency of
    the CUDA-graph launch with L2 warm (launches back to back) and cold (a 2x L2 write
    before every launch, timed apart from it)."""
    import flowgen as fg
    reg = fg.registry_c1()
    rec = fg.window_records_c1(reg)
    n = rec["srcaddr"].size
    ctx = gnm.Context(device=local, window_slots=4)
    ctx.load(reg)
    dev = gnm.Records.to_device(rec)
    tune = ctx.autotune(dev, [0, n], [1])  # the library's launch shape for this window size
    plan = ctx.plan(dev, [0, n], [1])
    stream = torch.cuda.current_stream()
    for _ in range(20):
        plan.launch(stream)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        plan.launch(stream)
    b.record(stream)
    torch.cuda.synchronize()
    warm_us = a.elapsed_time(b) * 1e3 / reps
    flush = torch.empty(2 * 129 * (1 << 20) // 4, dtype=torch.int32, device=f"cuda:{local}")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps // 10)]
    for e0, e1 in ev:
        flush.fill_(1)
        e0.record(stream)
        plan.launch(stream)
        e1.record(stream)
    torch.cuda.synchronize()
    cold_us = float(np.mean([e0.elapsed_time(e1) for e0, e1 in ev])) * 1e3
    plan.close()
    ctx.close()
    # the same window with per-flow rate statistics (histograms, min, max) kept as well
    ctx = gnm.Context(device=local, window_slots=4, rate_stats=1)
    ctx.load(reg)
    ctx.autotune(dev, [0, n], [1])
    plan = ctx.plan(dev, [0, n], [1])
    for _ in range(20):
        plan.launch(stream)
    a.record(stream)
    for _ in range(reps):
        plan.launch(stream)
    b.record(stream)
    torch.cuda.synchronize()
    rs_us = a.elapsed_time(b) * 1e3 / reps
    plan.close()
    ctx.close()
    return {"workload": f"one window of {n:,} records; {reg.n_sites} sites / {reg.n:,} prefixes (registry in "
                        "shared memory); CUDA-graph launch",
            "warm_us": warm_us, "warm_records_per_s": n / (warm_us * 1e-6), "warm_reps": reps,
            "cold_us": cold_us, "cold_records_per_s": n / (cold_us * 1e-6), "cold_reps": len(ev),
            "cold": "a 258 MB write (2x L2) before every timed launch",
            "warm_us_with_rate_stats": rs_us,
            "rate_stats": "per-flow 10 kb/s histograms (1,000 keys x 10,001 buckets, cleared every launch), "
                          "least and greatest rate",
            "tuned": {"block_threads": tune.block_threads, "ctas_per_sm": tune.ctas_per_sm, "unroll": tune.unroll,
                      "default_us": round(tune.default_ms * 1e3, 2), "tuned_us": round(tune.best_ms * 1e3, 2)}}


E2E_HOST = {"auto": "read in place by the kernels over the host link",
            "in_place": "read in place by the kernels over the host link",
            "stage": "copied to a device staging buffer, then processed",
            "pipeline": "chunks of windows copied on a second stream, each processed as soon as it "
                        "has landed"}
AGGREGATIONS = {"auto": 0, "direct": 1, "warp": 2}  # gnm_aggregation


def parse_shape(text):
    """'k=v,k=v' -> {k: int(v)} (context config fields of a fixed launch shape)."""
    out = {}
    for item in filter(None, (t.strip() for t in text.split(","))):
        k, v = item.split("=")
        out[k.strip()] = int(v)
    return out


def agg_times(tune):
    """The autotuner's fastest candidate per aggregation: per-lane shared-memory atomics
    (direct) against one atomic per distinct key of a warp (warp)."""
    return {"direct": round(tune.best_ms_by_agg[1], 4) or None, "warp": round(tune.best_ms_by_agg[2], 4) or None}


def batched_c4(gnm, torch, local, steps, warmup, aggregation=0):
    """256 uneven windows (lognormal sizes around 200,000 records, clamped to 10,000-2,000,000)
    over the 500-site registry in one CUDA-graph launch, shape autotuned by the library."""
    import flowgen as fg
    reg = fg.registry_c1()
    counts = fg.uneven_windows_c4()
    rec, off = fg.batched_records_c4(reg, counts)
    n, n_win = int(off[-1]), len(off) - 1
    dev = gnm.Records.to_device(rec)
    del rec
    ctx = gnm.Context(device=local, window_slots=n_win + 8, aggregation=aggregation)
    ctx.load(reg)
    ids = np.arange(n_win, dtype=np.uint64)
    tune = ctx.autotune(dev, off, ids)
    plan = ctx.plan(dev, off, ids, kernel_times=True)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        plan.launch(stream)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    a.record(stream)
    for _ in range(steps):
        plan.launch(stream)
    b.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    ms = a.elapsed_time(b) / steps
    plan.launch(stream)
    kms = {k: round(v, 4) for k, v in plan.kernel_times()}
    info = ctx.registry_info()
    alg = 24 * n + n_win * (2 * reg.n_sites * (48 + 8 + 1) + 4 * 48) + int(info.n_ranges) * 8
    peak, peak_kind = hbm_peak()
    gbs = alg / (ms / 1e3) / 1e9
    plan.close()
    ctx.close()
    return {"workload": f"{n_win} windows, {n:,} records (lognormal sizes, median 200,000, clamped "
                        f"10,000-2,000,000); {reg.n_sites} sites / {reg.n:,} prefixes -> {int(info.n_ranges):,} "
                        f"ranges (registry in shared memory); one CUDA-graph launch",
            "records_per_s": n / (ms / 1e3), "ms": ms, "achieved_gbs": gbs, "frac": gbs / peak,
            "peak_kind": peak_kind, "kernels_ms": kms,
            "tuned": {"block_threads": tune.block_threads, "unroll": tune.unroll, "aggregation": tune.aggregation,
                      "radix_bits": tune.radix_bits,
                      "placement": tune.placement, "ctas_per_sm": tune.ctas_per_sm,
                      "best_ms_by_aggregation": agg_times(tune)}}


def serve_c5(gnm, torch, local, speedup=1000.0, realtime_minutes=10, pool_n=20_000_000, budget=4 << 30,
             n_random=10, sat_minutes=120):
    """Streaming replay of the 24-hour schedule: Poisson batch arrivals (1,000-500,000
    records, 1e6 records/s on average times the diurnal factor) over the learned-index
    100,000-site registry, one window per minute (1,440 windows), closed at the minute's
    end. Host batches (pinned) are cut at random offsets of a pool. Reports:
    - the whole day replayed `speedup` times faster than real time: p50/p99 window latency
      over the 1,440 windows (window close -> rates and flags final on the device); every
      60th window and `n_random` random ones are also processed alone from the same batches
      and must be bit-identical to their results in the mix;
    - the `sat_minutes` around the daily peak submitted as fast as possible;
    - `realtime_minutes` around the peak at real time (x1)."""
    import flowgen as fg
    reg = fg.registry_c3()
    pool = fg.make_records(reg, pool_n, seed=4, p_reg=0.9, zipf_s=0.9)
    pinned = {k: torch.from_numpy(np.ascontiguousarray(pool[k]).view(np.int32)).pin_memory() for k in gnm.FIELDS}
    hpool = {k: v.numpy().view(np.uint32) for k, v in pinned.items()}
    dpool = {k: v.cuda() for k, v in pinned.items()}
    t_all, sz_all = fg.serving_schedule_c5(hours=24.0)
    rng = np.random.default_rng(5)
    off_all = rng.integers(0, pool_n - sz_all + 1)
    day_min = 24 * 60
    checked = sorted(set(range(0, day_min, 60)) | set(rng.choice(day_min, n_random, replace=False).tolist()))
    ctx = gnm.Context(device=local, window_slots=16)
    ctx.load(reg)
    keys = torch.from_numpy(fg.lookup_keys_c3(reg, 10_000_000).view(np.int32)).cuda()
    ctx.rmi_train(keys, root_kind=gnm.ROOT_LINEAR, n_leaves=4096, leaf_iters=4)
    got = {}
    queued = []

    def part(t0, minutes):
        sel = (t_all >= t0) & (t_all < t0 + minutes * 60.0)
        tt = t_all[sel] - t0
        return tt, sz_all[sel], off_all[sel], (tt // 60.0).astype(np.int64)

    def replay(srv, speedup, base, sched, minutes, keep=()):
        """Submits a schedule (speedup None: as fast as possible); window w has id base + w;
        the results of the windows in `keep` are read when they are reported."""
        times, sizes, offs, win_of = sched
        reports = []
        queued.clear()

        def take(rs):
            for r in rs:
                reports.append(r)
                queued.append(r[4])
                if r[0] - base in keep:
                    got[r[0] - base] = ctx.dense(r[0])
        nb, bi, wc = len(times), 0, 0
        start = time.perf_counter()
        if speedup is None:  # as fast as possible: the schedule in submit_many calls of 512 events
            ev_b, ev_c, ev_w, ev_f = [], [], [], []
            while bi < nb or wc < minutes:
                if bi < nb and times[bi] <= (wc + 1) * 60.0:
                    ev_b.append(int(offs[bi])), ev_c.append(int(sizes[bi]))
                    ev_w.append(base + int(win_of[bi])), ev_f.append(0)
                    bi += 1
                else:
                    ev_b.append(0), ev_c.append(0), ev_w.append(base + wc), ev_f.append(1)
                    wc += 1
            start = time.perf_counter()
            for k in range(0, len(ev_b), 512):
                srv.submit_many(pool_recs, ev_b[k:k + 512], ev_c[k:k + 512], ev_w[k:k + 512], ev_f[k:k + 512])
                take(srv.poll(queued=True))
            take(srv.poll(wait_all=True, queued=True))
            return reports, time.perf_counter() - start
        while bi < nb or wc < minutes:
            now = (time.perf_counter() - start) * speedup
            ta = times[bi] if bi < nb else float("inf")
            tc = (wc + 1) * 60.0
            if min(ta, tc) <= now:
                if ta <= tc:
                    a = int(offs[bi])
                    srv.submit(gnm.Records({k: v[a:a + int(sizes[bi])] for k, v in hpool.items()}),
                               base + int(win_of[bi]))
                    bi += 1
                else:
                    srv.close_window(base + wc)
                    wc += 1
            take(srv.poll(queued=True))
        take(srv.poll(wait_all=True, queued=True))
        return reports, time.perf_counter() - start

    def pct(v, q):
        return float(np.percentile(v, q, method="inverted_cdf")) if len(v) else None

    pool_recs = gnm.Records(hpool)
    day = part(0.0, day_min)
    peak = part(6 * 3600.0 - sat_minutes * 30.0, sat_minutes)
    rt = part(6 * 3600.0 - realtime_minutes * 30.0, realtime_minutes) if realtime_minutes else None
    with gnm.Stream(ctx, budget_bytes=budget, n_cuda_streams=4) as srv:
        # warm-up window (not reported): first use of the kernels and the arena
        srv.submit(gnm.Records({k: v[:100_000] for k, v in hpool.items()}), 1 << 40, close=True)
        srv.poll(wait_all=True)
        torch.cuda.synchronize()
        reports, wall = replay(srv, speedup, 0, day, day_min, keep=set(checked))
        q_ms = list(queued)
        st = srv.stats()
        sat_reports, sat_wall = replay(srv, None, 1 << 20, peak, sat_minutes)
        sat_st = srv.stats()
        rt_reports, rt_wall = replay(srv, 1.0, 1 << 21, rt, realtime_minutes) if rt else ([], 0.0)
    # the checked windows processed alone (open, the same batches from a device copy of the
    # pool, close) must give the same results as in the mix
    ok = True
    times, sizes, offs, win_of = day
    for w in checked:
        wid = (1 << 41) + w
        ctx.open(wid)
        for i in np.nonzero(win_of == w)[0]:
            a, n = int(offs[i]), int(sizes[i])
            ctx.add(gnm.Records({k: v[a:a + n] for k, v in dpool.items()}), wid)
        ctx.close_window(wid)
        ast, aun, arate, afl = ctx.dense(wid)
        gst, gun, grate, gfl = got[w]
        ok = ok and (np.array_equal(gst, ast) and np.array_equal(gun, aun) and np.array_equal(gfl, afl)
                     and np.array_equal(grate, arate, equal_nan=True))
    ctx.close()
    lat = [r[2] for r in reports if r[3] == 0]
    n_rec = int(sizes.sum())
    sat_lat = [r[2] for r in sat_reports if r[3] == 0]
    rt_lat = [r[2] for r in rt_reports if r[3] == 0]
    n_sat = int(peak[1].sum())
    out = {"workload": f"the 24-hour schedule: {day_min} one-minute windows, {len(times):,} Poisson batches of "
                       f"1,000-500,000 records ({n_rec:,} records, 1e6 records/s x (1 + 0.7 sin(2 pi t / 1 day)) "
                       f"on average), replayed x{speedup:g} faster than real time; {reg.n_sites:,}-site "
                       f"learned-index registry (4,096 minimax leaves); host batches from a pinned "
                       f"{pool_n:,}-record pool",
           "records_per_s": n_rec / wall, "offered_records_per_s": n_rec / (day_min * 60.0 / speedup),
           "wall_s": wall, "windows": len(lat),
           "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "max_ms": max(lat) if lat else None,
           "latency": "window close -> rates and flags final (host clock)",
           "slowest_windows_ms": sorted(((r[2], r[0], r[4]) for r in reports if r[3] == 0), reverse=True)[:3],
           "queued_p50_ms": pct(q_ms, 50), "queued_p99_ms": pct(q_ms, 99),
           "queued": "closing submit -> finalisation enqueued (host side of the latency)",
           "budget_bytes": budget, "peak_inflight_bytes": int(st["peak_inflight_bytes"]),
           "batches": int(st["batches"]), "batches_queued": int(st["batches_queued"]),
           "checked_windows": checked, "mix_equals_alone": bool(ok),
           "check": "each checked window processed alone from the same batches, bit-identical to its result "
                    "in the mix (the same windows are checked against the oracle by the full-size tests)",
           "saturated": {"workload": f"the {sat_minutes} minutes around the daily peak ({n_sat:,} records)",
                         "records_per_s": n_sat / sat_wall, "wall_s": sat_wall,
                         "h2d_gbs": 24 * n_sat / sat_wall / 1e9,
                         "p50_ms": pct(sat_lat, 50), "p99_ms": pct(sat_lat, 99),
                         "peak_inflight_bytes": int(sat_st["peak_inflight_bytes"]),
                         "batches_queued": int(sat_st["batches_queued"] - st["batches_queued"]),
                         "note": "submitted as fast as possible (gnm_stream_submit_many, 512 batches or closes "
                                 "per call); latency includes the queue behind the budget"}}
    if rt:
        out["realtime"] = {"workload": f"the {realtime_minutes} minutes around the daily peak at real time "
                                       f"(x1, {int(rt[1].sum()):,} records in {len(rt[0]):,} batches)",
                           "wall_s": rt_wall, "windows": len(rt_lat), "p50_ms": pct(rt_lat, 50),
                           "p99_ms": pct(rt_lat, 99), "max_ms": max(rt_lat) if rt_lat else None}
    return out


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


def cpu_oracle_c3(cores, n=5_000_000):
    """The oracle on a sample of the learned-index workload (100,000-site registry): one
    window of n records on all host threads; records/s (scaled from the sample)."""
    import flowgen as fg
    import oracle
    reg = fg.registry_c3()
    rec = fg.make_records(reg, n, seed=2, p_reg=0.9, zipf_s=0.9)
    lpm = oracle.LPM(reg.prefix, reg.plen, reg.site)
    t0 = time.perf_counter()
    st, _ = oracle.window(lpm, reg.local_prefix, reg.local_len, reg.n_sites, rec, n_threads=cores)
    oracle.flags(st, oracle.rates(st), 1e8)
    t = time.perf_counter() - t0
    return {"value": n / t, "unit": "records/s", "cores": cores,
            "sample": f"one window of {n:,} records (the learned-index registry), {t:.2f} s"}


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
    ap.add_argument("--no-learned", action="store_true", help="skip the plain-vs-learned index comparison")
    ap.add_argument("--no-serve", action="store_true", help="skip the streaming-server replay")
    ap.add_argument("--only", default="all", choices=["all", "learned", "serve", "batched", "window", "paper"],
                    help="run one leg alone (profiling): the learned-index comparison, the server replay "
                         "or the batched windows")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-window batched launch")
    ap.add_argument("--aggregation", default="auto", choices=list(AGGREGATIONS),
                    help="per-key reduction of the hour and batched workloads (auto: the autotuner's choice)")
    ap.add_argument("--shape", default="",
                    help="launch shape of the hour workload instead of autotuning it, as context config "
                         "fields (e.g. block_threads=1024,unroll=1,radix_bits=13,split=2,key_directory=3): "
                         "profiles then capture the kernels the plain run timed")
    ap.add_argument("--e2e-host", default="auto", choices=["auto", "stage", "in_place", "pipeline"],
                    help="how the end-to-end leg's page-locked host records reach the kernels "
                         "(gnm_config.host_records)")
    ap.add_argument("--e2e-streams", type=int, default=2,
                    help="compute streams that consecutive end-to-end steps alternate between")
    ap.add_argument("--learned-records", type=int, default=50_000_000)
    ap.add_argument("--learned-modes", default="bsearch,radix,rmi,rmi_mse,rmi65536")
    ap.add_argument("--serve-speedup", type=float, default=1000.0,
                    help="time compression of the 24-hour serving replay")
    ap.add_argument("--serve-realtime-minutes", type=int, default=10,
                    help="minutes of the real-time (x1) serving slice (0: none)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch

    import flowgen as fg
    from paper_1108_1785_gb300 import build, gnm

    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    build.build()
    if args.only != "all":  # one leg alone, for profiling; prints its own JSON object
        if args.only == "learned":
            leg = learned_vs_plain(gnm, torch, local, args.steps, args.warmup, args.learned_records,
                                   tuple(args.learned_modes.split(",")))
        elif args.only == "batched":
            leg = batched_c4(gnm, torch, local, args.steps, args.warmup, AGGREGATIONS[args.aggregation])
        elif args.only == "window":
            leg = window_c1(gnm, torch, local)
        elif args.only == "paper":
            leg = paper_lookup(gnm, torch, local, args.steps, args.warmup)
        else:
            leg = serve_c5(gnm, torch, local, speedup=args.serve_speedup, realtime_minutes=args.serve_realtime_minutes)
        print(json.dumps({"leg": args.only, **leg}), flush=True)
        return 0
    reg = fg.registry_c2()
    rec, off = fg.hour_records_c2(reg, seed=1 + rank)
    n = int(off[-1])
    n_win = len(off) - 1
    shape = parse_shape(args.shape)
    ctx = gnm.Context(device=local, window_slots=2 * n_win + 8,
                      **{"aggregation": AGGREGATIONS[args.aggregation],
                         "host_records": getattr(gnm, "HOST_" + args.e2e_host.upper()), **shape})
    ctx.load(reg)
    dev = gnm.Records.to_device(rec)
    ids = np.arange(n_win, dtype=np.uint64)
    # the library's own autotuner picks block size, records per thread, aggregation and
    # registry placement on this workload (outside the timed region), unless the launch
    # shape is given
    tune = None if shape else ctx.autotune(dev, off, ids)
    info = ctx.registry_info()
    plan = ctx.plan(dev, off, ids)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        plan.launch(stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches = 0
    # the clock samples (every 200 ms) cover the timed steps plus about 0.5 s of identical
    # untimed steps on each side of them, so that they see the GPU under this load
    pad = int(min(20000, max(1, 500.0 / max(tune.best_ms if tune else 0.2, 1e-3))))
    with ClockSampler(local) as clk:
        for _ in range(pad):
            plan.launch(stream)
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
        for _ in range(pad):
            plan.launch(stream)
        torch.cuda.synchronize()
    total_ms = ev[0][0].elapsed_time(ev[-1][1])
    step_ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    total_ms = max_over_ranks(total_ms, world)
    value = n * world * args.steps / (total_ms / 1e3)
    clocks = clk.summary()
    clocks["window"] = f"timed steps plus {pad} identical untimed steps before and after them"

    # per-kernel device durations: the same graph with timing events between its kernels,
    # launched K more times on the same stream
    plan.close()
    tplan = ctx.plan(dev, off, ids, kernel_times=True)
    for _ in range(args.warmup):
        tplan.launch(stream)
    per = []
    for _ in range(args.steps):
        tplan.launch(stream)
        per.append(tplan.kernel_times())
    tplan.close()
    names = [k for k, _ in per[0]]
    kern_avg = {nm: float(np.mean([p[i][1] for p in per])) for i, nm in enumerate(names)}

    # algorithmic bytes: 24 B per record read, each window's per-key sums (48 B), rate
    # (8 B) and flag (1 B) written once, the registry read once -- split over the kernels
    # as the method's own compulsory reads and writes each one performs. The 4-byte key a
    # split launch passes from its key kernel to its aggregation kernel is the design's own
    # traffic, not the method's: it is not counted (it shows in traffic_ratio).
    nk = 2 * reg.n_sites
    out_bytes = n_win * (nk * (48 + 8 + 1) + 4 * 48)
    reg_bytes = int(info.n_ranges) * 8
    alg_bytes = 24 * n + out_bytes + reg_bytes
    if names == ["k_aggregate"]:  # fused: the one kernel does it all
        kern_bytes = {"k_aggregate": alg_bytes}
    else:
        kern_bytes = {"k_keys": 8 * n + reg_bytes,                       # the two addresses, the registry
                      "k_aggregate": 16 * n + (0 if "k_finalize_windows" in names else out_bytes),
                      "k_finalize_windows": out_bytes}
    top = max(kern_avg, key=kern_avg.get)
    peak, peak_kind = hbm_peak()
    achieved = kern_bytes[top] / (kern_avg[top] / 1e3) / 1e9
    step_gbs = alg_bytes / (step_ms / 1e3) / 1e9
    traffic = None
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
        if t.get("kernel_source_hash") == kernel_source_hash() and t.get("records") == n:
            traffic = t["dram_bytes_per_launch"].get(top)
    except Exception:
        pass

    out = {
        "metric": METRIC, "value": value, "unit": "records/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": workload_desc(n, n_win, reg, int(info.n_ranges)),
                   "global_batch": n * world, "windows_per_step": n_win * world,
                   "parallelism": f"replicas x{world} (independent hours per GPU)",
                   "lookup": LOOKUP_NAMES.get(int(info.lookup_mode), str(int(info.lookup_mode))),
                   "l2": "inputs 240 MB per GPU > 129 MB L2; no flush between steps",
                   "launch": f"CUDA graph per step: {launches // max(1, args.steps)} kernel launches "
                             "(per-record site keys, persistent per-window aggregation, per-window finalise)"
                             if launches // max(1, args.steps) == 3 else
                             f"CUDA graph per step: {launches // max(1, args.steps)} kernel launch(es)",
                   "tuned": {"block_threads": tune.block_threads, "ctas_per_sm": tune.ctas_per_sm,
                             "unroll": tune.unroll, "aggregation": tune.aggregation, "placement": tune.placement,
                             "radix_bits": tune.radix_bits, "split": tune.split, "key_directory": tune.key_directory,
                             "keys_unroll": tune.keys_unroll,
                             "default_ms": round(tune.default_ms, 4), "tuned_ms": round(tune.best_ms, 4),
                             "best_ms_by_aggregation": agg_times(tune), "candidates": tune.n_tried}
                   if tune else {"fixed": shape}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                     "traffic_ratio": (traffic / kern_bytes[top]) if traffic else None,
                     "kernel": top, "kernel_ms": kern_avg[top], "algorithmic_bytes": kern_bytes[top],
                     "kernels_ms": kern_avg,
                     # every kernel of the step on its own method bytes (the key and aggregation
                     # kernels take similar times, so either can be the dominant one in a run)
                     "kernels_frac": {k: kern_bytes[k] / (kern_avg[k] / 1e3) / 1e9 / peak for k in kern_avg},
                     "kernel_timing": "CUDA events between the graph's kernels, K further launches",
                     "step": {"ms": step_ms, "algorithmic_bytes": alg_bytes, "achieved": step_gbs,
                              "frac": step_gbs / peak}},
        "clocks": clocks,
        "gpu_launches": launches,
    }

    if not args.no_e2e:
        # end to end through the C ABI: page-locked host records (the kernels read them in
        # place over the host link) -> D2H of every window's full result: the six u64 sums
        # per (site, dir) key, the unmatched classes, the rates and the flags
        pinned = {k: torch.from_numpy(np.ascontiguousarray(rec[k]).view(np.int32)).pin_memory()
                  for k in gnm.FIELDS}
        hostrec = gnm.Records({k: v.numpy() for k, v in pinned.items()})

        def host(n_items, dt):
            t = torch.empty(n_items * np.dtype(dt).itemsize, dtype=torch.uint8).pin_memory()
            return t.numpy().view(dt)

        # two sets of window ids and result buffers: a step's results are copied out on a
        # second stream while the next step (the other set) is processed
        outs = [(host(n_win * nk * 6, np.uint64), host(n_win * 4 * 6, np.uint64), host(n_win * nk, np.float64),
                 host(n_win * nk, np.uint8)) for _ in range(2)]
        sets = [ids + n_win, ids + 2 * n_win]
        copy_stream = torch.cuda.Stream()
        # consecutive steps alternate between compute streams (each step's windows and the
        # library's launch buffers are its own), so that one step's device-only work (its
        # finalisation, kernel ramps) overlaps the next step's reads over the host link
        comp = [stream] + [torch.cuda.Stream() for _ in range(max(1, args.e2e_streams) - 1)]

        def e2e_step(k):
            ctx.process_windows(hostrec, off, sets[k % 2], comp[k % len(comp)])
            ctx.windows_results_async(sets[k % 2], *outs[k % 2], stream=copy_stream)

        for k in range(max(2, args.warmup)):
            e2e_step(k)
        copy_stream.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            e2e_step(k)
        copy_stream.synchronize()
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, world)
        # the host link: a plain copy of the same page-locked records (best of three)
        dst = {k: torch.empty_like(v, device=f"cuda:{local}") for k, v in pinned.items() if k in gnm.FIELDS}
        best = None
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for k in dst:
                dst[k].copy_(pinned[k], non_blocking=True)
            b.record(stream)
            b.synchronize()
            best = a.elapsed_time(b) if best is None else min(best, a.elapsed_time(b))
        h2d_gbs = sum(v.numel() * v.element_size() for v in dst.values()) / (best / 1e3) / 1e9
        del dst
        out["e2e"] = {"value": n * world * args.steps / e2e_s, "unit": "records/s",
                      "h2d_bytes_per_step": 24 * n, "d2h_bytes_per_step": n_win * (nk * (48 + 8 + 1) + 4 * 48),
                      "api": "gnm_windows_process over page-locked host records (host_records "
                             f"{args.e2e_host.upper()}: " + E2E_HOST[args.e2e_host] + ") + "
                             "gnm_windows_results_async (sums, unmatched classes, rates, flags) on a second "
                             "stream, overlapping the next step's processing; two sets of window ids alternate"
                             + (f", consecutive steps on {len(comp)} compute streams" if len(comp) > 1 else ""),
                      "h2d_copy_gbs": h2d_gbs,
                      "records_bound": h2d_gbs * 1e9 / 24,
                      "bound_note": "a plain copy of the step's page-locked records to the device, timed "
                                    "in the same run; at 24 bytes a record it bounds e2e"}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        s = cpu_oracle_hour(reg, rec, off, cores)
        # one thread (the paper's CPU baseline ran on one core) on the first 10 windows
        off10 = off[:11]
        s1 = cpu_oracle_hour(reg, {k: v[:int(off10[-1])] for k, v in rec.items()}, off10, 1)
        out["cpu_baseline"] = {"value": n / s, "unit": "records/s", "cores": cores, "kind": "oracle",
                               "sample": f"the whole step once: {n_win} windows, {n:,} records "
                                         f"({s:.2f} s on {cores} threads)",
                               "single_thread": {"value": int(off10[-1]) / s1, "unit": "records/s",
                                                 "sample": f"first 10 windows, {int(off10[-1]):,} records, 1 thread"},
                               "learned_registry": cpu_oracle_c3(cores)}
    ctx.close()
    del dev
    if world == 1 and not args.no_learned:
        out["learned_index"] = learned_vs_plain(gnm, torch, local, args.steps, args.warmup, args.learned_records,
                                                tuple(args.learned_modes.split(",")))
    if world == 1 and not args.no_batched:
        out["window"] = window_c1(gnm, torch, local)
        out["paper_lookup"] = paper_lookup(gnm, torch, local, args.steps, args.warmup)
        out["batched"] = batched_c4(gnm, torch, local, args.steps, args.warmup, AGGREGATIONS[args.aggregation])
    if world == 1 and not args.no_serve:
        out["serving"] = serve_c5(gnm, torch, local, speedup=args.serve_speedup,
                                  realtime_minutes=args.serve_realtime_minutes)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
