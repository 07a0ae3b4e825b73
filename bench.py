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
    """Digest of the scan kernel's source and of the file that configures its launches
    (tile size, grid, the context's L2 fetch limit)."""
    h = hashlib.sha256()
    for name in ("scan_kernel.cuh", "mdrq.cu"):
        h.update(open(os.path.join(ROOT, "paper_1801_03644_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def dram_traffic_per_launch(workload: str, alg_bytes_per_launch: float):
    """DRAM bytes per scan launch from the committed ncu summary of a smaller case of this
    workload (same recipe, fewer rows and queries), scaled to this run's launch by the
    captured launch's DRAM bytes / early-break algorithmic bytes (``early_break_bytes``);
    None when the summary is missing, counts other bytes, or the kernel source changed
    since it was taken."""
    p = os.path.join(ROOT, "profiles", "mdrq_scan_kernel_%s.traffic.json" % workload)
    if not os.path.exists(p):
        return None, None
    d = json.load(open(p))
    if d.get("scan_kernel_digest") != scan_kernel_digest() or "early_break_bytes" not in d:
        return None, None
    ratio = float(d["dram_bytes"]) / float(d["early_break_bytes"])
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


# ----------------------------------------------------------------------------- answers

def same_answers(off_a, ids_a, off_b, ids_b) -> bool:
    """Identical CSR answers: the same per-query offsets and the same ids (device
    tensors compared in full)."""
    import torch
    off_a, off_b = np.asarray(off_a), np.asarray(off_b)
    if not np.array_equal(off_a, off_b):
        return False
    total = int(off_a[-1])
    return bool(torch.equal(ids_a[:total], ids_b[:total]))


def verify_with_oracle(columns, queries, ids, off, which, nthreads: int) -> dict:
    """Count and ids of the queries ``which`` against the CPU oracle (evaluated one
    dimension at a time, Sec. 3.2; pinned on its own in the test suite). ``ids`` is
    the batch's device answer (CSR by ``off``)."""
    import oracle
    oracle.build()
    off = np.asarray(off, dtype=np.int64)
    t0 = time.perf_counter()
    bad = []
    for q in which:
        a, b = int(off[q]), int(off[q + 1])
        want = oracle.mdrq_columnwise(columns, queries[q], nthreads=nthreads)
        have = ids[a:b].cpu().numpy().view(np.uint32) if b > a else np.zeros(0, np.uint32)
        if have.size != want.size or not np.array_equal(have, want):
            bad.append(int(q))
    return {"queries": len(which), "of": len(queries), "mismatches": len(bad), "first_mismatches": bad[:8],
            "oracle": "CPU oracle, dimension at a time, %d threads" % nthreads,
            "seconds": time.perf_counter() - t0}


def zone_candidates(table, cols_dev, n: int, tile: int = 4096, max_runs: int = 1024):
    """For the tile pruning of zone maps: a function of a query plan that gives the row
    mask of the tiles the scan visits. A tile is a candidate when, for every predicate
    whose column's zone map is in use (``mdrq_zone_map_info``), the tile's [min, max]
    meets the interval; more than ``max_runs`` runs of candidates are visited as one
    span from the first to the last. The tiles' min and max are computed here from the
    columns, independently of the library's zone maps."""
    import torch
    ntiles = (n + tile - 1) // tile
    pad = ntiles * tile - n
    used, tmin, tmax = {}, {}, {}
    for j, x in enumerate(cols_dev):
        used[j] = table.zone_map_info(j)["used"]
        if used[j]:
            xp = torch.cat([x, x[-1:].expand(pad)]) if pad else x
            tmin[j] = xp.view(ntiles, tile).amin(dim=1)
            tmax[j] = xp.view(ntiles, tile).amax(dim=1)

    def visited(plan):
        cand = torch.ones(ntiles, dtype=torch.bool, device=cols_dev[0].device)
        for (j, lo, hi) in plan:
            if used[j]:
                lo_t = torch.tensor(lo, dtype=cols_dev[j].dtype, device=cand.device)
                hi_t = torch.tensor(hi, dtype=cols_dev[j].dtype, device=cand.device)
                cand &= (tmax[j] >= lo_t) & (tmin[j] <= hi_t)
        starts = cand.clone()
        starts[1:] &= ~cand[:-1]
        if int(starts.sum()) > max_runs:
            idx = torch.nonzero(cand).flatten()
            cand[int(idx[0]):int(idx[-1]) + 1] = True
        return cand.repeat_interleave(tile)[:n]
    return visited


def early_break_bytes(table, cols_dev, queries, n: int, granule: int = 32, visited=None):
    """Algorithmic bytes of the plain scan of ``queries`` with its early break (Sec.
    2.2.4) at DRAM-sector granularity: for each query, in the order the scan evaluates
    its predicates (``mdrq_explain_query``), 32 B for every 32-byte sector (8 rows) of
    the column that still holds a row satisfying all earlier predicates, plus 4 B per
    answer id (``granule``: the same count at a coarser fetch size, for comparison with
    the DRAM traffic; ``visited``: a function of the plan giving the rows the scan
    reaches at all, for tile pruning). Counted on the GPU with plain tensor operations, outside any timed
    region; it does not depend on the kernel (two lanes of 4 rows share a sector, and
    a lane whose rows have all failed issues no load)."""
    import torch
    rows = granule // 4
    pad = (-n) % rows
    total = 0.0
    for q in queries:
        empty, plan = table.explain(q)
        if empty:
            continue
        alive = visited(plan) if visited is not None else None
        for (j, lo, hi) in plan:
            x = cols_dev[j]
            if alive is None:
                sectors = (n + rows - 1) // rows
            else:
                a = torch.cat([alive, alive.new_zeros(pad)]) if pad else alive
                sectors = int(a.view(-1, rows).any(dim=1).sum())
            total += float(granule) * sectors
            lo_t = torch.tensor(lo, dtype=x.dtype, device=x.device)
            hi_t = torch.tensor(hi, dtype=x.dtype, device=x.device)
            m = (x >= lo_t) & (x <= hi_t)
            alive = m if alive is None else alive & m
        total += 4.0 * (n if alive is None else int(alive.sum()))
    return total


def d2h_gbs(torch, nbytes: int = 1 << 30) -> float:
    """Device-to-pinned-host copy rate of one large copy (CUDA events), for context."""
    src = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    dst = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    dst.copy_(src, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        dst.copy_(src, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    return 3 * nbytes / (e0.elapsed_time(e1) / 1e3) / 1e9


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


def learned_leg(args, table, enc, step, nq, total_ids, world, barrier, stream, ids, ids_ref, off_ref, cells=None):
    """Learned range narrower (PLA, the MLP-rooted two-stage model, and no model: the
    whole key column searched) and zone-map tile pruning on a Z-sorted table: queries/s
    and speedup over the plain scan of the same batch with zone maps off (every tile
    read), model error, window coverage and the keys the window searches read. ``step`` answers the batch into
    ``ids``; every leg's answer must equal the reference answer (``off_ref``,
    ``ids_ref``) id for id."""
    import torch
    from paper_1801_03644_gb300 import mdrq, shards

    def timed(mode, zones):
        table.set_batch_mode(mode)
        table.set_zone_maps(zones)
        for _ in range(args.warmup):
            step()
        ids.fill_(-1)
        ms, off = timed_steps(torch, stream, step, args.steps, barrier)
        ms = shards.max_over_ranks(ms)
        return world * nq * args.steps / (ms / 1e3), ms / args.steps, same_answers(off_ref, ids_ref, off, ids)

    base, base_ms, same_b = timed(mdrq.BATCH_PLAIN, mdrq.ZONES_OFF)
    zval, zms, same_z = timed(mdrq.BATCH_PLAIN, mdrq.ZONES_AUTO)
    zrows, ztiles = table.zone_scan_info()
    out = {"plain_no_zone_maps": {"value": base, "unit": UNIT, "ms_per_step": base_ms,
                                  "answers_identical_to_plain": same_b},
           "zone_pruned_plain": {"value": zval, "unit": UNIT, "ms_per_step": zms,
                                 "speedup_vs_plain": zval / base, "rows_visited_per_query": zrows / nq,
                                 "tiles_visited": ztiles, "answers_identical_to_plain": same_z}}
    for name, model in (("pla", mdrq.MODEL_PLA), ("mlp", mdrq.MODEL_MLP), ("none", mdrq.MODEL_NONE)):
        info = table.learn([0, 1, 2, 3], model, cells=cells)
        lvalue, lms, same_l = timed(mdrq.BATCH_LEARNED, mdrq.ZONES_AUTO)
        rows, widen = table.learn_window_rows()
        ranges, probes = table.learn_search_info()
        # dense-equivalent bytes: 16 per window row (the four key columns) plus the ids;
        # the scan's early break reads fewer, so this is not a DRAM figure
        lbytes = 16.0 * rows + 4.0 * total_ids
        out[name] = {"value": lvalue, "unit": UNIT, "ms_per_step": lms,
                     "window_effective_gbs": lbytes / (lms / 1e3) / 1e9,
                     "window_effective_frac": lbytes / (lms / 1e3) / 1e9 / measured_peaks()["hbm_gbs"],
                     "effective_rule": "dense equivalent, not bytes moved: 16 B per window row plus 4 B per id",
                     "speedup_vs_plain": lvalue / base, "speedup_vs_zone_pruned": lvalue / zval,
                     "max_error_rows": info["max_error"],
                     "segments": info["segments"], "train_ms": info["train_ms"],
                     "window_rows_per_query": rows / nq, "window_widenings": widen,
                     "key_ranges": ranges, "search_keys_read_per_range": probes / max(1, ranges),
                     "answers_identical_to_plain": same_l}
        if name == "pla":
            v0, ms0, same0 = timed(mdrq.BATCH_LEARNED, mdrq.ZONES_OFF)
            out[name]["without_zone_maps"] = {"value": v0, "ms_per_step": ms0,
                                              "answers_identical_to_plain": same0}
    table.set_batch_mode(mdrq.BATCH_PLAIN)
    table.set_zone_maps(mdrq.ZONES_AUTO)
    return out


def learned_workload_leg(args, world, barrier):
    """The learned narrower on the 2e8 x 4 Z-sorted table with 4096 queries, against
    the plain scan of the same batch; a seeded sample of the answers against the CPU
    oracle (the test suite compares all 4096)."""
    import torch
    from paper_1801_03644_gb300 import mdrq
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

    off_ref = step()
    torch.cuda.synchronize()
    ids_ref = ids[:total].clone()
    nq = len(wl.queries)
    res = {"workload": wl.name, "recipe": wl.recipe, "unit": UNIT, "answer_ids_per_step": total}
    res.update(learned_leg(args, table, enc, step, nq, total, world, barrier, stream, ids, ids_ref, off_ref,
                           cells=wl.key_bounds))
    table.close()
    del ids
    if not args.no_verify:
        pick = np.sort(np.random.default_rng(4).choice(nq, size=min(args.verify_sample, nq), replace=False))
        res["verified"] = verify_with_oracle(wl.columns, wl.queries, ids_ref, off_ref, pick.tolist(),
                                             os.cpu_count() or 1)
        res["verified"]["sample"] = "seeded sample of the batch; the test suite compares every query"
    del ids_ref
    torch.cuda.empty_cache()
    return res


def small_table_leg(args, world, barrier):
    """The 1,000,000 x 3 uniform table (12 MB of columns, 100 queries of about 1%
    selectivity), kernel time only (the scan's own CUDA events, bracketing each launch
    on its stream):

    * warm: the batch of 100 queries in one persistent launch, repeated; the table stays
      in the 126 MB L2 between launches (the hot-cache convention of Sec. 7.1.2), so
      this measures the scan out of L2, not HBM;
    * cold: each query in a launch of its own, after a 512 MB read-and-write of a
      scratch buffer that evicts the table from L2 (outside the events), so that the
      launch reads its columns from HBM.

    Byte rates use the early-break algorithmic bytes (``early_break_bytes``) and the
    dense bytes (every row of every constrained column); fractions are of the measured
    HBM copy peak and of the nominal 7.9 TB/s."""
    import torch
    from paper_1801_03644_gb300 import mdrq, shards
    wl = W.uniform_small()
    cols = [torch.from_numpy(c).cuda() for c in wl.columns]
    t = mdrq.Table(cols)
    t.set_batch_mode(mdrq.BATCH_PLAIN)
    enc = t.encode_batch(wl.queries)
    probe = torch.empty(1, dtype=torch.int32, device="cuda")
    st, off = t.query_batch_raw(enc, probe.data_ptr(), 0, True)
    ids = torch.empty(max(1, int(off[-1])), dtype=torch.int32, device="cuda")
    nq = len(wl.queries)
    peak = measured_peaks()["hbm_gbs"]

    def step():
        st, o = t.query_batch_raw(enc, ids.data_ptr(), ids.numel(), True)
        if st != mdrq.OK:
            raise mdrq.MDRQError(st, "mdrq_query_batch")
        return o

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    t.scan_timing(True)
    t.scan_timing_read(reset=True)
    for _ in range(args.steps):
        off = step()
    warm = t.scan_timing_read(reset=True)
    ids_batch = ids[: int(off[-1])].clone()
    least = early_break_bytes(t, cols, wl.queries, wl.n)
    dense = warm["bytes"] / max(1, warm["scan_launches"])
    warm_s = shards.max_over_ranks(warm["ms"]) / 1e3 / max(1, warm["scan_launches"])

    # cold: one launch per query, L2 evicted before each
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    out = torch.empty(wl.n, dtype=torch.int32, device="cuda")
    match = True
    cold_ms = 0.0
    launches = 0
    for _ in range(args.steps):
        for q, query in enumerate(wl.queries):
            flush.add_(1)
            torch.cuda.synchronize()
            t.scan_timing_read(reset=True)
            one = t.query(query, out=out)
            tm = t.scan_timing_read(reset=True)
            cold_ms += tm["ms"]
            launches += tm["scan_launches"]
            match = match and bool(torch.equal(one, ids_batch[int(off[q]):int(off[q + 1])]))
    t.scan_timing(False)
    del flush
    cold_s = shards.max_over_ranks(cold_ms) / 1e3 / max(1, launches)
    least_q, dense_q = least / nq, dense / nq
    res = {
        "workload": wl.name, "recipe": wl.recipe, "unit": UNIT,
        "early_break_bytes_per_query": least_q, "dense_bytes_per_query": dense_q,
        "warm": {"value": world * nq / warm_s, "unit": UNIT, "kernel_ms_per_batch": warm_s * 1e3,
                 "launches": warm["scan_launches"],
                 "early_break_gbs": least / warm_s / 1e9, "dense_gbs": dense / warm_s / 1e9,
                 "early_break_frac": least / warm_s / 1e9 / peak,
                 "dense_frac": dense / warm_s / 1e9 / peak,
                 "dense_frac_of_nominal": dense / warm_s / 1e9 / NOMINAL_HBM_GBS,
                 "served_from": "L2 (12 MB table; the batch's 100 queries re-read it)"},
        "cold": {"value": world / cold_s, "unit": UNIT, "kernel_us_per_query": cold_s * 1e6,
                 "launches": launches,
                 "early_break_gbs": least_q / cold_s / 1e9, "dense_gbs": dense_q / cold_s / 1e9,
                 "early_break_frac": least_q / cold_s / 1e9 / peak,
                 "dense_frac": dense_q / cold_s / 1e9 / peak,
                 "dense_frac_of_nominal": dense_q / cold_s / 1e9 / NOMINAL_HBM_GBS,
                 "cache": "L2 evicted by a 512 MB read-and-write before every launch (outside the events)",
                 "answers_identical_to_batch": match},
        "peak_gbs": peak, "nominal_peak_gbs": NOMINAL_HBM_GBS,
    }
    res["verified"] = verify_with_oracle(wl.columns, wl.queries, ids_batch, off, list(range(nq)),
                                         os.cpu_count() or 1)
    t.close()
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
    verify_every = 64
    served = []
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

        kept = {}  # a sample of the served answers (1 in verify_every), checked afterwards

        def consumer():
            done = 0
            while done < count:
                while state["n"] <= done:
                    time.sleep(1e-4)
                upto = min(state["n"], done + 256)
                sample = [i for i in range(done, upto) if i % verify_every == 0]
                _, _, lat = srv.wait_many(tickets[done:upto], release=not sample)
                if sample:
                    for i in sample:
                        st, d_ids, cnt, _ = srv.wait(int(tickets[i]))
                        kept[i] = (st, d_ids.cpu().numpy().view(np.uint32) if d_ids is not None
                                   else np.zeros(0, np.uint32))
                    for i in range(done, upto):
                        srv.release(int(tickets[i]))
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
        served.extend((i, st_, a) for i, (st_, a) in kept.items())
    sys.setswitchinterval(switch)
    table.close()
    res = {"workload": wl.name, "recipe": wl.recipe, "result_memory_cap_bytes": 2 << 30,
           "arrivals": "open-loop Poisson", "rates": rows}
    if not args.no_verify:
        # the kept answers of the timed runs against the CPU oracle
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        bad = []
        for i, st_, a in served:
            want = oracle.mdrq_columnwise(wl.columns, wl.queries[i], nthreads=os.cpu_count() or 1)
            if st_ != mdrq.OK or a.size != want.size or not np.array_equal(a, want):
                bad.append(i)
        res["verified"] = {"queries": len(served), "mismatches": len(bad), "first_mismatches": bad[:8],
                           "sample": "every %d-th served answer of each timed rate, copied out before its "
                                     "release; the test suite compares all 20,000 queries" % verify_every,
                           "oracle": "CPU oracle, dimension at a time", "seconds": time.perf_counter() - t0}
    return res


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
    nthreads = os.cpu_count() or 1

    def barrier():
        if world > 1:
            dist.barrier()

    stream = torch.cuda.current_stream()
    # the columns are made resident once (not timed); the table refers to them in place
    cols_dev = [torch.from_numpy(c).cuda() for c in wl.columns]
    table = mdrq.Table(cols_dev)
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
        off_ref = step()
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
    # the timed batch's answer: every other leg must reproduce it id for id
    ids_ref = ids[:total_ids].clone()

    # ---- the same plain batch replayed as a prepared CUDA graph (no per-call host work)
    def graph_steps(mode):
        table.set_batch_mode(mode)
        ids.fill_(-1)
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
                "answers_identical_to_plain": same_answers(off_ref, ids_ref, off_g, ids)}

    plain_graph = graph_steps(mdrq.BATCH_PLAIN)
    table.set_batch_mode(mdrq.BATCH_PLAIN)

    # ---- batched shared scan (the same batch, answers identical): speedup over plain
    batched = None
    if not args.no_batched:
        table.set_batch_mode(mdrq.BATCH_SHARED)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        ids.fill_(-1)
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
                   "mode": "shared scan: each constrained column encoded once per batch into 16-bit "
                           "codes, per-row query sets of each chunk of up to 128 queries from "
                           "elementary-interval tables looked up by code, two passes (count, write)",
                   "answers_identical_to_plain": same_answers(off_ref, ids_ref, off_b, ids)}
        # the same batch with the values searched per chunk instead of encoded once
        table.set_shared_codes(False)
        for _ in range(args.warmup):
            step()
        ids.fill_(-1)
        vms, off_v = timed_steps(torch, stream, step, args.steps, barrier)
        vms = shards.max_over_ranks(vms)
        batched["values_searched"] = {"value": world * nq * args.steps / (vms / 1e3), "unit": UNIT,
                                      "ms_per_step": vms / args.steps,
                                      "answers_identical_to_plain": same_answers(off_ref, ids_ref, off_v, ids)}
        table.set_shared_codes(True)
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
        # the shared scan's bound: HBM for the least bytes a batch needs (every
        # constrained column once per chunk of queries, plus the ids)
        cols = len({p[0] for q in wl.queries for p in q})
        least_bytes = 4.0 * wl.n * cols + 4.0 * total_ids
        for leg in (batched, tuned):
            t_s = leg["ms_per_step"] / 1e3
            leg["hbm_frac_least_bytes"] = least_bytes / t_s / 1e9 / measured_peaks()["hbm_gbs"]
        batched["bounds"] = {"least_bytes_per_batch": least_bytes,
                             "least_bytes_rule": "every column some query constrains, read once, plus 4 B per id"}
        table.set_batch_mode(mdrq.BATCH_PLAIN)

    # ---- learned range narrower: on this table when it is Z-sorted, else on its own
    learned = None
    if args.workload == "zorder_learned":
        learned = learned_leg(args, table, enc, step, nq, total_ids, world, barrier, stream, ids, ids_ref, off_ref,
                              cells=wl.key_bounds)

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

        def e2e_run(host_mode):
            table.set_host_answers(host_mode)
            for _ in range(max(1, args.warmup)):
                step_host()
            barrier()
            torch.cuda.synchronize()
            table.scan_timing(True)
            table.scan_timing_read(reset=True)
            t0 = time.perf_counter()
            for _ in range(args.steps):
                off_h = step_host()
            torch.cuda.synchronize()
            barrier()
            secs = shards.max_over_ranks(time.perf_counter() - t0)
            kern = table.scan_timing_read(reset=True)
            table.scan_timing(False)
            back = host_ids[:total_ids].to("cuda")
            same = same_answers(off_ref, ids_ref, off_h, back)
            del back
            return secs, kern, same

        e2e_s, e2e_kernel, same_d = e2e_run(mdrq.HOST_AUTO)
        st_s, st_kernel, same_s = e2e_run(mdrq.HOST_STAGED)
        di_s, di_kernel, same_di = e2e_run(mdrq.HOST_DIRECT)
        table.set_host_answers(mdrq.HOST_AUTO)
        auto_copies = e2e_kernel["scan_launches"] > args.steps  # AUTO took the staged copies
        npreds = sum(len(q) for q in wl.queries)
        e2e = {"value": world * nq * args.steps / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": 16 * npreds + 16 * nq,
               "d2h_bytes_per_step": 8 * (nq + 1) + 4 * total_ids,
               "wall_ms_per_step": 1e3 * e2e_s / args.steps,
               "scan_kernel_ms_per_step": e2e_kernel["ms"] / args.steps,
               "launches_per_step": e2e_kernel["scan_launches"] / args.steps,
               "answers_identical_to_plain": same_d,
               "path": ("mdrq_query_batch with host query descriptors and a pinned host answer "
                        "buffer (MDRQ_HOST_AUTO: %s); host wall clock" %
                        ("the batch's plain output is staged, so the ids are staged in device memory "
                         "and each launch's are copied out on a second stream while the next runs"
                         if auto_copies else "the scan writes the ids itself over the CPU-GPU link")),
               "bytes": "h2d: the host descriptors passed to the call (16 B per predicate and per "
                        "query; the library stages them as one copy of 16 B per query and 32 B per "
                        "kept predicate); d2h: the offsets and every id",
               "staged": {"value": world * nq * args.steps / st_s, "unit": UNIT,
                          "wall_ms_per_step": 1e3 * st_s / args.steps,
                          "scan_kernel_ms_per_step": st_kernel["ms"] / args.steps,
                          "launches_per_step": st_kernel["scan_launches"] / args.steps,
                          "d2h_gbs_one_copy_alone": d2h_gbs(torch),
                          "answers_identical_to_plain": same_s,
                          "path": "the same call with the ids staged in device memory and copied "
                                  "out per launch on a second stream (mdrq_set_host_answers STAGED)"},
               "direct": {"value": world * nq * args.steps / di_s, "unit": UNIT,
                          "wall_ms_per_step": 1e3 * di_s / args.steps,
                          "scan_kernel_ms_per_step": di_kernel["ms"] / args.steps,
                          "launches_per_step": di_kernel["scan_launches"] / args.steps,
                          "answers_identical_to_plain": same_di,
                          "path": "the same call with the ids written into the pinned buffer by the "
                                  "kernels over the CPU-GPU link (mdrq_set_host_answers DIRECT; with "
                                  "staged output the ordering pass writes them, after the scan)"}}
        del host_ids

    # ---- roofline of the scan kernel: bytes / event-timed launch duration
    peaks = measured_peaks()
    launches = max(1, timing["scan_launches"])
    dense_per_launch = timing["bytes"] / launches
    dense_rule = "4 B per row per constrained column (every row of the table) plus 4 B per id"
    if zone_rows is not None:
        # every constrained column of every row of the tiles left, plus the ids
        cols = max(len({p[0] for p in q}) for q in wl.queries)
        dense_per_launch = 4.0 * cols * zone_rows + 4.0 * total_ids
        dense_rule = ("4 B per row per constrained column over the rows of the tiles the zone "
                      "maps leave (%d rows per query) plus 4 B per id" % (zone_rows // max(1, nq)))
    avg_launch_s = timing["ms"] / 1e3 / launches
    # a staged plain launch counts four kernels: the scan and the ordering pass's three
    staged_output = args.workload != "zorder_learned" and timing["kernel_launches"] == 4 * launches
    vis = zone_candidates(table, cols_dev, wl.n) if zone_rows is not None else None
    alg_per_launch = early_break_bytes(table, cols_dev, wl.queries, wl.n, visited=vis)
    alg64_per_launch = early_break_bytes(table, cols_dev, wl.queries, wl.n, granule=64, visited=vis)
    alg_rule = ("early-break bytes: per query, in the scan's predicate order, 32 B per 32-byte "
                "sector (8 rows) of each evaluated column that still holds a row satisfying "
                "the earlier predicates, plus 4 B per id")
    if zone_rows is not None:
        alg_rule += "; rows of the tiles the zone maps rule out are never reached"
    achieved = alg_per_launch / avg_launch_s / 1e9 if avg_launch_s > 0 else 0.0
    effective = dense_per_launch / avg_launch_s / 1e9 if avg_launch_s > 0 else 0.0
    traffic, ratio = dram_traffic_per_launch(args.workload, alg_per_launch)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"],
                "traffic": traffic,
                "peak_source": peaks["source"] + " (HBM copy bandwidth)",
                "kernel": ("mdrq_scan_window_kernel (plain batch over the tiles the zone maps leave)"
                           if args.workload == "zorder_learned" else
                           "mdrq_scan_staged_kernel (plain batch, staged output; the three kernels of "
                           "the ordering pass run after it, inside the step but outside this timing)"
                           if staged_output else "mdrq_scan_kernel"),
                "alg_bytes_per_launch": alg_per_launch, "alg_bytes_rule": alg_rule,
                "avg_launch_ms": avg_launch_s * 1e3,
                "ordering_pass_ms_per_step": (ms / args.steps - avg_launch_s * 1e3) if staged_output else 0.0,
                "scan_launches": timing["scan_launches"],
                "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "nominal_peak": NOMINAL_HBM_GBS,
                "traffic_over_alg_bytes": ratio,
                "dram_gbs_moved": traffic / avg_launch_s / 1e9 if traffic and avg_launch_s > 0 else None,
                "dram_frac_moved": (traffic / avg_launch_s / 1e9 / peaks["hbm_gbs"]
                                    if traffic and avg_launch_s > 0 else None),
                "early_break_bytes_64B_fetches": alg64_per_launch,
                "effective_gbs": effective, "effective_frac": effective / peaks["hbm_gbs"],
                "effective_rule": "dense equivalent, not bytes moved: " + dense_rule}

    # ---- every answer of the timed batch against the CPU oracle (rank 0)
    verified = None
    if rank == 0 and not args.no_verify:
        verified = verify_with_oracle(wl.columns, wl.queries, ids_ref, off_ref, list(range(nq)), nthreads)

    # ---- CPU baseline: the oracle as it stands, on the host cores (rank 0, N = 1)
    cpu = None
    if world == 1 and rank == 0 and not args.no_cpu_baseline:
        m, secs = time_oracle(wl, args.cpu_seconds, nthreads)
        cpu = {"value": m / secs, "unit": UNIT, "cores": nthreads, "kind": "oracle",
               "sample": "first %d of the %d queries, whole table (%d rows), %d threads over "
                         "contiguous horizontal partitions, object at a time" % (m, nq, wl.n, nthreads),
               "host_cpu": host_cpu_model()}
        # the same scan on one thread, the same queries from the first (a shorter sample)
        m1, secs1 = time_oracle(wl, args.cpu_seconds / 3.0, 1, min_queries=1)
        cpu["single_thread"] = {"value": m1 / secs1, "unit": UNIT, "cores": 1,
                                "sample": "first %d of the %d queries, whole table, 1 thread" % (m1, nq)}

    # ---- the small table, the learned narrower and the server, each on its own table
    table.close()
    del ids, ids_ref, cols_dev
    torch.cuda.empty_cache()
    small = None
    if args.workload != "uniform_1M" and not args.no_small:
        small = small_table_leg(args, world, barrier)
    if args.workload != "zorder_learned" and not args.no_learned:
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
            "cpu_baseline": cpu, "verified": verified,
            "answer_ids_per_step": total_ids, "achieved_selectivity": selectivity,
            "plain_graph": plain_graph, "batched": batched, "small_table": small,
            "learned": learned, "serving": serving,
        }), flush=True)


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
    ap.add_argument("--no-verify", action="store_true", help="skip the oracle check of the timed batch")
    ap.add_argument("--no-small", action="store_true", help="skip the 1M x 3 warm / cold leg")
    ap.add_argument("--only-small", action="store_true",
                    help="run the 1M x 3 warm / cold leg alone (a profiling case)")
    ap.add_argument("--verify-sample", type=int, default=256,
                    help="queries of the Z-sorted batch checked against the oracle")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.only_small:
        # profiling case: the 1M x 3 table's warm and cold launches alone
        import torch
        torch.cuda.set_device(local_rank)
        print(json.dumps({"small_table": small_table_leg(args, 1, lambda: None)}), flush=True)
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
