#!/usr/bin/env python
"""Benchmark of the GB300 MDRQ scan: queries/s and scan GB/s against the HBM roofline.

A step answers one batch of multidimensional range queries (Sec. 2.1) over a table
resident on the GPU, through the C ABI (``mdrq_query_batch``), with every answer
written to device memory as an ascending id list. The default workload is a
100,000,000 x 8 float32 table (4 uniform columns, 4 columns of a 20-cluster Gaussian
mixture) and a batch of 1024 partial-match queries on 2..8 dimensions with target
selectivity log-uniform in [1e-5, 0.2]. The 3.2 GB of columns exceed the 126 MB L2,
so steps need no cache flush between them.

Prints one JSON line (rank 0). ``--impl reference`` times the CPU oracle instead.
Launch with N > 1 through torch.distributed.run: every rank answers its own batch on
its own GPU (independent replicas, weak scaling); the timed region is bracketed by
barriers and the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1801_03644_gb300 import workloads as W  # noqa: E402

METRIC = "MDRQ queries/s"
UNIT = "queries/s"


def make_workload(name: str, rows=None, queries=None):
    """The named workload at its full size, or at ``rows`` rows with the first ``queries``
    queries (smaller cases of the same recipe, for profiling)."""
    kw = {}
    if rows:
        kw["n"] = int(rows)
    if name == "mixed_clustered":
        wl = W.mixed_clustered(**kw)
    elif name == "uniform_1M":
        wl = W.uniform_small(**kw)
    elif name == "skewed_mixed":
        wl = W.skewed_mixed_types(**kw)
    elif name == "zorder_learned":
        wl = W.zorder_learned(**kw)
    else:
        raise SystemExit("unknown workload %s" % name)
    if queries and int(queries) < len(wl.queries):
        wl.queries = wl.queries[: int(queries)]
        wl.recipe += "; the first %d of them" % int(queries)
    return wl


def workload_config(wl, name: str) -> dict:
    return {"workload": wl.name, "n": wl.n, "d": wl.d, "queries_per_step": len(wl.queries),
            "recipe": wl.recipe,
            "cache": ("inputs larger than L2: no flush between steps"
                      if 4 * wl.n * wl.d > 126e6 else
                      "table fits in L2: hot cache as in Sec. 7.1.2, L2 not flushed"),
            "answers": "ascending uint32 id lists in device memory (CSR)",
            "parallelism": "replicas"}


# ----------------------------------------------------------------------------- clocks

CLOCK_FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
                "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
                "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]


class ClockSampler:
    """nvidia-smi sampling every 200 ms while the timed region runs."""

    def __init__(self, gpu_id: str):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + ",".join(CLOCK_FIELDS), "--format=csv,noheader,nounits",
                 "-i", gpu_id, "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) != len(CLOCK_FIELDS):
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def gpu_smi_id(torch, dev: int) -> str:
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev)


# ----------------------------------------------------------------------------- peaks, traffic

NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def scan_kernel_digest() -> str:
    src = os.path.join(ROOT, "paper_1801_03644_gb300", "csrc", "scan_kernel.cuh")
    return hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]


def dram_traffic_per_launch(workload: str, alg_bytes_per_launch: float):
    """DRAM bytes per scan launch from the committed ncu summary of this workload, scaled
    to this run's average launch by the captured launches' traffic / algorithmic ratio;
    None when the summary is missing or the kernel source changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "mdrq_scan_kernel_%s.traffic.json" % workload)
    if not os.path.exists(p):
        return None, None
    d = json.load(open(p))
    if d.get("scan_kernel_digest") != scan_kernel_digest():
        return None, None
    ratio = float(d["dram_bytes"]) / float(d["algorithmic_bytes"])
    return ratio * alg_bytes_per_launch, ratio


def selectivity_summary(offsets, n: int) -> dict:
    """Achieved selectivity of a batch's queries (answer size / rows), from the batch's
    CSR offsets (nq + 1 entries); the recipes only target a selectivity (Sec. 2.1: on
    correlated dimensions the product of per-dimension shares misses it)."""
    counts = np.diff(np.asarray(offsets, dtype=np.int64))
    out = {"queries": int(counts.size)}
    if counts.size == 0 or n <= 0:
        return out
    sel = counts / float(n)
    out.update({"mean": float(sel.mean()), "median": float(np.median(sel)), "min": float(sel.min()),
                "max": float(sel.max()), "empty_queries": int((counts == 0).sum())})
    return out


# ----------------------------------------------------------------------------- oracle timing

def time_oracle(wl, budget_s: float, nthreads: int, min_queries: int = 2):
    """Answer the batch's queries in order with the CPU oracle until ``budget_s`` has
    passed; returns (queries answered, seconds)."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    done = 0
    for q in wl.queries:
        oracle.mdrq(wl.columns, q, nthreads=nthreads)
        done += 1
        if done >= min_queries and time.perf_counter() - t0 > budget_s:
            break
    return done, time.perf_counter() - t0


def host_cpu_model() -> str:
    """The host CPU's model name as lscpu prints it (the machine the oracle runs on)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def run_reference(args, rank: int, world: int) -> None:
    """The CPU oracle on the host cores: each step a bounded sample of the same batch."""
    if rank != 0:
        return
    wl = make_workload(args.workload, args.rows, args.queries)
    nthreads = os.cpu_count() or 1
    # size the sample so that one step takes about --cpu-seconds
    m, secs = time_oracle(wl, args.cpu_seconds, nthreads)
    sample = wl.queries[:m]
    sub = W.Workload(wl.name, wl.columns, sample, wl.recipe)
    for _ in range(max(0, args.warmup - 1)):
        time_oracle(sub, 1e9, nthreads, min_queries=m)
    times = []
    for _ in range(args.steps):
        _, s = time_oracle(sub, 1e9, nthreads, min_queries=m)
        times.append(s)
    total = sum(times)
    value = m * args.steps / total
    cfg = workload_config(wl, args.workload)
    desc = "first %d of the %d queries per step, whole table (%d rows)" % (m, len(wl.queries), wl.n)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                         "sample": desc, "host_cpu": host_cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ----------------------------------------------------------------------------- GPU arm

def timed_steps(torch, stream, step, steps, barrier):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    last = None
    for _ in range(steps):
        last = step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    return e0.elapsed_time(e1), last


def learned_leg(args, table, enc, step, nq, total_ids, world, barrier, stream):
    """Learned range narrower (PLA and MLP) and zone-map tile pruning on a Z-sorted table:
    queries/s and speedup over the plain scan of the same batch with zone maps off
    (every tile read), model error and window coverage."""
    import torch
    from paper_1801_03644_gb300 import mdrq, shards

    def timed(mode, zones):
        table.set_batch_mode(mode)
        table.set_zone_maps(zones)
        for _ in range(args.warmup):
            step()
        ms, off = timed_steps(torch, stream, step, args.steps, barrier)
        ms = shards.max_over_ranks(ms)
        return world * nq * args.steps / (ms / 1e3), ms / args.steps, off

    base, base_ms, off_b = timed(mdrq.BATCH_PLAIN, mdrq.ZONES_OFF)
    zval, zms, off_z = timed(mdrq.BATCH_PLAIN, mdrq.ZONES_AUTO)
    zrows, ztiles = table.zone_scan_info()
    out = {"plain_no_zone_maps": {"value": base, "unit": UNIT, "ms_per_step": base_ms,
                                  "answers_identical_to_plain": bool(int(off_b[-1]) == total_ids)},
           "zone_pruned_plain": {"value": zval, "unit": UNIT, "ms_per_step": zms,
                                 "speedup_vs_plain": zval / base, "rows_visited_per_query": zrows / nq,
                                 "tiles_visited": ztiles,
                                 "answers_identical_to_plain": bool(int(off_z[-1]) == total_ids)}}
    for name, model in (("pla", mdrq.MODEL_PLA), ("mlp", mdrq.MODEL_MLP)):
        info = table.learn([0, 1, 2, 3], model)
        lvalue, lms, off_l = timed(mdrq.BATCH_LEARNED, mdrq.ZONES_AUTO)
        rows, widen = table.learn_window_rows()
        # bytes as the learned narrower's roofline counts them: 16 per window row (the
        # four key columns) plus the ids
        lbytes = 16.0 * rows + 4.0 * total_ids
        out[name] = {"value": lvalue, "unit": UNIT, "ms_per_step": lms,
                     "window_gbs": lbytes / (lms / 1e3) / 1e9,
                     "window_frac": lbytes / (lms / 1e3) / 1e9 / measured_peaks()["hbm_gbs"],
                     "speedup_vs_plain": lvalue / base, "speedup_vs_zone_pruned": lvalue / zval,
                     "max_error_rows": info["max_error"],
                     "segments": info["segments"], "train_ms": info["train_ms"],
                     "window_rows_per_query": rows / nq, "window_widenings": widen,
                     "answers_identical_to_plain": bool(int(off_l[-1]) == total_ids)}
        if name == "pla":
            v0, ms0, _ = timed(mdrq.BATCH_LEARNED, mdrq.ZONES_OFF)
            out[name]["without_zone_maps"] = {"value": v0, "ms_per_step": ms0}
    table.set_batch_mode(mdrq.BATCH_PLAIN)
    table.set_zone_maps(mdrq.ZONES_AUTO)
    return out


def learned_workload_leg(args, world, barrier):
    """The learned narrower on the 2e8 x 4 Z-sorted table with 4096 queries, against
    the plain scan of the same batch."""
    import torch
    from paper_1801_03644_gb300 import mdrq, shards
    wl = make_workload("zorder_learned", args.learned_rows)
    stream = torch.cuda.current_stream()
    table = mdrq.Table(wl.columns)
    table.set_batch_mode(mdrq.BATCH_PLAIN)
    enc = table.encode_batch(wl.queries)
    probe = torch.empty(1, dtype=torch.int32, device="cuda")
    st, off = table.query_batch_raw(enc, probe.data_ptr(), 0, True)
    total = int(off[-1])
    ids = torch.empty(max(1, total), dtype=torch.int32, device="cuda")

    def step():
        st, o = table.query_batch_raw(enc, ids.data_ptr(), ids.numel(), True)
        if st != mdrq.OK:
            raise mdrq.MDRQError(st, "mdrq_query_batch")
        return o

    nq = len(wl.queries)
    res = {"workload": wl.name, "recipe": wl.recipe, "unit": UNIT, "answer_ids_per_step": total}
    res.update(learned_leg(args, table, enc, step, nq, total, world, barrier, stream))
    table.close()
    return res


def serving_leg(args):
    """Open-loop Poisson arrivals into the continuous-batching server on the 2e7 x 16
    table: per arrival rate, throughput and p50 / p99 latency (submit to answer, and
    from the scheduled arrival). The load generator submits, in one call, every query
    whose arrival time has come; a consumer thread waits for the answers in submission
    order, in chunks, and releases them."""
    import threading
    from paper_1801_03644_gb300 import mdrq
    wl = W.serving_table(n=args.serving_rows, nq=20_000)
    table = mdrq.Table(wl.columns)
    rows = []
    # the load generator and the consumer are Python threads: hand the interpreter lock
    # over often, so that a submission is not held back behind the other thread
    switch = sys.getswitchinterval()
    sys.setswitchinterval(1e-4)
    import gc
    for rate in args.serving_rates:
        count = int(min(len(wl.queries), max(500, rate * args.serving_seconds)))
        arrivals = np.asarray(W.poisson_arrivals(rate, count, seed=int(rate)))
        enc = table.encode_batch(wl.queries[:count])
        descs, keep, _ = enc
        srv = mdrq.Server(table, result_bytes=2 << 30, max_batch=512)
        tickets = np.zeros(count, dtype=np.uint64)
        submitted_at = np.zeros(count)  # seconds after t0
        lat_us = np.zeros(count)
        state = {"n": 0, "last": None}

        def consumer():
            done = 0
            while done < count:
                while state["n"] <= done:
                    time.sleep(1e-4)
                upto = min(state["n"], done + 256)
                _, _, lat = srv.wait_many(tickets[done:upto], release=True)
                lat_us[done:upto] = lat
                done = upto
            state["last"] = time.perf_counter()

        th = threading.Thread(target=consumer)
        gc.collect()
        gc.disable()  # no collector pause inside the load generator's schedule
        th.start()
        t0 = time.perf_counter()
        i = 0
        while i < count:
            now = time.perf_counter() - t0
            if arrivals[i] > now:
                time.sleep(min(arrivals[i] - now, 1e-3))
                continue
            j = int(np.searchsorted(arrivals, now, side="right"))
            sub = ctypes_array_slice(descs, i, j)
            tk = srv.submit_batch((sub, keep[i:j], j - i))
            submitted_at[i:j] = time.perf_counter() - t0
            tickets[i:j] = tk
            state["n"] = j
            i = j
        th.join()
        gc.enable()
        span = state["last"] - t0
        stats = srv.stats()
        srv.stop()
        # latency: the server's (submit to answer), and from the scheduled arrival (plus
        # the time the query waited for the load generator's submission call)
        pct = lambda a, q: float(a[min(a.size - 1, int(q * (a.size - 1) + 0.5))])
        lat = np.sort(lat_us / 1e3)
        lat_arr = np.sort(lat_us / 1e3 + (submitted_at - arrivals) * 1e3)
        rows.append({"offered_qps": rate, "queries": count, "throughput_qps": count / span,
                     "p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99),
                     "p50_from_arrival_ms": pct(lat_arr, 0.5), "p99_from_arrival_ms": pct(lat_arr, 0.99),
                     "batches": stats["batches"], "deferred": stats["deferred"]})
    sys.setswitchinterval(switch)
    table.close()
    return {"workload": wl.name, "recipe": wl.recipe, "result_memory_cap_bytes": 2 << 30,
            "arrivals": "open-loop Poisson", "rates": rows}


def ctypes_array_slice(arr, i: int, j: int):
    """A view of elements [i, j) of a ctypes array (no copy)."""
    import ctypes
    elem = arr._type_
    return (elem * max(1, j - i)).from_buffer(arr, i * ctypes.sizeof(elem))


def run_gpu(args, rank: int, world: int, local_rank: int) -> None:
    import torch
    import torch.distributed as dist
    from paper_1801_03644_gb300 import mdrq, shards

    torch.cuda.set_device(local_rank)
    dev = torch.cuda.current_device()
    wl = make_workload(args.workload, args.rows, args.queries)
    if world > 1 and rank > 0:
        # each rank answers its own batch: same table recipe, queries from a rank stream
        qrng = W.rng_for(1000 + rank, 1)
        samples = W.quantile_samples(wl.columns, W.rng_for(1000 + rank, 2))
        dtypes = [c.dtype for c in wl.columns]
        qs = []
        for q0 in wl.queries:
            dims = [p[0] for p in q0]
            s = W.log_uniform(qrng, 1e-5, 0.2)
            qs.append(W.target_selectivity_query(samples, dtypes, dims, s, qrng))
        wl = W.Workload(wl.name, wl.columns, qs, wl.recipe)
    nq = len(wl.queries)

    stream = torch.cuda.current_stream()
    table = mdrq.Table(wl.columns)  # copied to the device once (not timed)
    table.set_batch_mode(mdrq.BATCH_PLAIN)  # the headline: every query scanned on its own
    enc = table.encode_batch(wl.queries)

    # first call sizes the answer buffer exactly
    probe = torch.empty(1, dtype=torch.int32, device="cuda")
    st, off = table.query_batch_raw(enc, probe.data_ptr(), 0, True)
    if st not in (mdrq.OK, mdrq.E_CAPACITY):
        raise mdrq.MDRQError(st, "mdrq_query_batch")
    total_ids = int(off[-1])
    selectivity = selectivity_summary(off, wl.n)
    ids = torch.empty(max(1, total_ids), dtype=torch.int32, device="cuda")

    def step():
        st, o = table.query_batch_raw(enc, ids.data_ptr(), ids.numel(), True)
        if st != mdrq.OK:
            raise mdrq.MDRQError(st, "mdrq_query_batch")
        return o

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- timed region: answers stay on the device
    sampler = ClockSampler(gpu_smi_id(torch, dev))
    time.sleep(0.3)
    table.scan_timing(True)
    table.scan_timing_read(reset=True)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    timing = table.scan_timing_read(reset=True)
    table.scan_timing(False)
    clocks = sampler.stop()
    # on the Z-sorted table the plain batch reads only the tiles its zone maps leave:
    # the rows of those tiles, as the last (the timed) launch visited them
    zone_rows = table.zone_scan_info()[0] if args.workload == "zorder_learned" else None
    ms = shards.max_over_ranks(ms)  # the slowest rank's time counts
    value = world * nq * args.steps / (ms / 1e3)

    # ---- a table that fits in L2: the same steps from a cold L2 (a 512 MB write before
    # every step, outside the timed span; each step timed on its own)
    cold = None
    if 4 * wl.n * wl.d <= 126e6:
        flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
        cold_ms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            step()
            c1.record(stream)
            torch.cuda.synchronize()
            cold_ms += c0.elapsed_time(c1)
        cold_ms = shards.max_over_ranks(cold_ms)
        alg_step = timing["bytes"] / max(1, timing["scan_launches"])
        cold = {"value": world * nq * args.steps / (cold_ms / 1e3), "unit": UNIT,
                "ms_per_step": cold_ms / args.steps,
                "algorithmic_gbs": alg_step / (cold_ms / args.steps / 1e3) / 1e9,
                "cache": "L2 flushed by a 512 MB write before every step; per-step CUDA events summed"}
        del flush

    # ---- the same plain batch replayed as a prepared CUDA graph (no per-call host work)
    def graph_steps(mode):
        table.set_batch_mode(mode)
        with table.prepare(wl.queries, out=ids) as p:
            for _ in range(args.warmup):
                p.launch()
            p.wait()
            barrier()
            g0 = torch.cuda.Event(enable_timing=True)
            g1 = torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            for _ in range(args.steps):
                p.launch()
            g1.record(stream)
            off_g = p.wait()
            barrier()
            gms = shards.max_over_ranks(g0.elapsed_time(g1))
            kernels = p.kernels()
        return {"value": world * nq * args.steps / (gms / 1e3), "unit": UNIT, "ms_per_step": gms / args.steps,
                "kernels_per_replay": kernels,
                "answers_identical_to_plain": bool(int(off_g[-1]) == total_ids)}

    plain_graph = graph_steps(mdrq.BATCH_PLAIN)
    table.set_batch_mode(mdrq.BATCH_PLAIN)

    # ---- batched shared scan (the same batch, answers identical): speedup over plain
    batched = None
    if not args.no_batched:
        table.set_batch_mode(mdrq.BATCH_SHARED)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        barrier()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for _ in range(args.steps):
            off_b = step()
        b1.record(stream)
        torch.cuda.synchronize()
        barrier()
        bms = shards.max_over_ranks(b0.elapsed_time(b1))
        bvalue = world * nq * args.steps / (bms / 1e3)
        batched = {"value": bvalue, "unit": UNIT, "ms_per_step": bms / args.steps,
                   "speedup_vs_plain": bvalue / value,
                   "mode": "shared scan: each constrained column read once per chunk of up to "
                           "128 queries, per-row query sets from elementary-interval tables, "
                           "two passes (count, write)",
                   "answers_identical_to_plain": bool(int(off_b[-1]) == total_ids)}
        # autotuned shape (untimed search), then the tuned batch as a prepared graph
        t_tune = time.perf_counter()
        tune = table.autotune(wl.queries)
        t_tune = time.perf_counter() - t_tune
        tuned = graph_steps(mdrq.BATCH_SHARED)
        tuned.update({"speedup_vs_plain": tuned["value"] / value, "unit_rows": tune["unit_rows"],
                      "image_kib": tune["image_kib"], "candidates": tune["candidates"],
                      "autotune_s": t_tune, "autotune_plain_ms": tune["plain_ms"],
                      "autotune_shared_default_ms": tune["shared_default_ms"],
                      "autotune_shared_best_ms": tune["shared_ms"],
                      "mode": "shared scan, autotuned shape (0 = built-in rule), replayed as a "
                              "prepared CUDA graph"})
        batched["tuned_graph"] = tuned
        # the shared scan's two bounds: ALU issue for the per-predicate work (two compares
        # and an AND per constrained value, rows x predicates x 3 simple operations at
        # SMs x 128 lanes x the SM clock), and HBM for the least bytes a batch needs
        # (every constrained column once, plus the ids)
        ops = 3.0 * wl.n * sum(len({p[0] for p in q}) for q in wl.queries)
        sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
        alu_peak = torch.cuda.get_device_properties(dev).multi_processor_count * 128 * sm_mhz * 1e6
        cols = len({p[0] for q in wl.queries for p in q})
        least_bytes = 4.0 * wl.n * cols + 4.0 * total_ids
        for leg in (batched, tuned):
            t_s = leg["ms_per_step"] / 1e3
            leg["alu_frac"] = ops / t_s / alu_peak
            leg["hbm_frac_least_bytes"] = least_bytes / t_s / 1e9 / measured_peaks()["hbm_gbs"]
        batched["bounds"] = {"ops_per_batch": ops, "alu_peak_ops_per_s": alu_peak,
                             "least_bytes_per_batch": least_bytes,
                             "note": "per-predicate operation count; the shared scan's own "
                                     "operations are interval lookups per column and chunk"}
        table.set_batch_mode(mdrq.BATCH_PLAIN)

    # ---- learned range narrower: on this table when it is Z-sorted, else on its own
    learned = None
    if args.workload == "zorder_learned":
        learned = learned_leg(args, table, enc, step, nq, total_ids, world, barrier, stream)

    # ---- end to end: host query descriptors in, host answers out (pinned)
    e2e = None
    if not args.no_e2e:
        host_ids = torch.empty(max(1, total_ids), dtype=torch.int32, pin_memory=True)
        hptr = host_ids.data_ptr()

        def step_host():
            st, o = table.query_batch_raw(enc, hptr, host_ids.numel(), False)
            if st != mdrq.OK:
                raise mdrq.MDRQError(st, "mdrq_query_batch")
            return o

        step_host()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step_host()
        torch.cuda.synchronize()
        barrier()
        e2e_s = time.perf_counter() - t0
        e2e_s = shards.max_over_ranks(e2e_s)
        npreds = sum(len(q) for q in wl.queries)
        e2e = {"value": world * nq * args.steps / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": 16 * npreds + 16 * nq,
               "d2h_bytes_per_step": 8 * (nq + 1) + 4 * total_ids,
               "path": "mdrq_query_batch with host query descriptors and a pinned host answer "
                       "buffer (each launch's ids copied while the next runs); host wall clock",
               "bytes": "h2d: the host descriptors passed to the call (16 B per predicate and per "
                        "query; the library stages them as one copy of 16 B per query and 32 B per "
                        "kept predicate); d2h: the offsets and every id"}

    # ---- roofline of the scan kernel (algorithmic bytes / event-timed duration)
    peaks = measured_peaks()
    launches = max(1, timing["scan_launches"])
    alg_per_launch = timing["bytes"] / launches
    bytes_rule = "4 B per row per constrained column (every row of the table) plus 4 B per id"
    if zone_rows is not None:
        # every constrained column of every row of the tiles left, plus the ids
        cols = max(len({p[0] for p in q}) for q in wl.queries)
        alg_per_launch = 4.0 * cols * zone_rows + 4.0 * total_ids
        bytes_rule = ("4 B per row per constrained column over the rows of the tiles the zone "
                      "maps leave (%d rows per query) plus 4 B per id" % (zone_rows // max(1, nq)))
    avg_launch_s = timing["ms"] / 1e3 / launches
    achieved = alg_per_launch / avg_launch_s / 1e9 if avg_launch_s > 0 else 0.0
    traffic, ratio = dram_traffic_per_launch(args.workload, alg_per_launch)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"],
                "traffic": traffic,
                "peak_source": peaks["source"] + " (HBM copy bandwidth)",
                "kernel": ("mdrq_scan_window_kernel (plain batch over the tiles the zone maps leave)"
                           if args.workload == "zorder_learned" else "mdrq_scan_kernel"),
                "alg_bytes_per_launch": alg_per_launch, "alg_bytes_rule": bytes_rule,
                "avg_launch_ms": avg_launch_s * 1e3,
                "scan_launches": timing["scan_launches"],
                "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                "dram_gbs_moved": traffic / avg_launch_s / 1e9 if traffic and avg_launch_s > 0 else None}

    # ---- CPU baseline: the oracle as it stands, on the host cores (rank 0, N = 1)
    cpu = None
    if world == 1 and rank == 0 and not args.no_cpu_baseline:
        nthreads = os.cpu_count() or 1
        m, secs = time_oracle(wl, args.cpu_seconds, nthreads)
        cpu = {"value": m / secs, "unit": UNIT, "cores": nthreads, "kind": "oracle",
               "sample": "first %d of the %d queries, whole table (%d rows), %d threads over "
                         "contiguous horizontal partitions" % (m, nq, wl.n, nthreads),
               "host_cpu": host_cpu_model()}
        # Listing 1 as written: one thread, the same queries from the first (a shorter sample)
        m1, secs1 = time_oracle(wl, args.cpu_seconds / 3.0, 1, min_queries=1)
        cpu["single_thread"] = {"value": m1 / secs1, "unit": UNIT, "cores": 1,
                                "sample": "first %d of the %d queries, whole table, 1 thread" % (m1, nq)}

    # ---- the learned narrower and the server, each on its own table
    if args.workload != "zorder_learned" and not args.no_learned:
        table.close()
        del ids
        torch.cuda.empty_cache()
        learned = learned_workload_leg(args, world, barrier)
    serving = None
    if not args.no_serving and world == 1:
        serving = serving_leg(args)

    if rank == 0:
        cfg = workload_config(wl, args.workload)
        cfg["mode"] = "plain scan: every query scanned on its own, the batch in one persistent launch"
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": cfg, "clocks": clocks, "e2e": e2e,
            "gpu_launches": timing["kernel_launches"], "roofline": roofline,
            "cpu_baseline": cpu, "answer_ids_per_step": total_ids, "achieved_selectivity": selectivity,
            "cold_l2": cold, "plain_graph": plain_graph,
            "batched": batched,
            "learned": learned, "serving": serving,
        }), flush=True)
    table.close()


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="mixed_clustered",
                    choices=["mixed_clustered", "uniform_1M", "skewed_mixed", "zorder_learned"])
    ap.add_argument("--rows", type=int, default=None,
                    help="smaller table of the same recipe (profiling cases)")
    ap.add_argument("--queries", type=int, default=None, help="first Q queries of the batch only")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the shared-scan measurement")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-narrower leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    ap.add_argument("--learned-rows", type=int, default=None)
    ap.add_argument("--serving-rows", type=int, default=20_000_000)
    ap.add_argument("--serving-rates", type=float, nargs="*", default=[1000.0, 10000.0, 100000.0])
    ap.add_argument("--serving-seconds", type=float, default=1.5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
