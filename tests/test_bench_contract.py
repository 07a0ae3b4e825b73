"""bench.py's output contract, checked on the CPU through its reference arm (the oracle
timed on a small sample): one JSON line with the keys the driver reads."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--rows", "100000",
                          "--queries", "8", "--steps", "2", "--warmup", "1", "--cpu-seconds", "0.1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == "MDRQ queries/s" and d["unit"] == "queries/s"
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1 and d["value"] > 0
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["config"]["workload"].startswith("mixed_clustered") and d["config"]["n"] == 100000
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["host_cpu"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_reference_arm_under_torchrun_prints_once():
    """Launched as the driver launches N > 1 (torchrun, one rank per GPU), the reference
    arm runs on rank 0 only and prints one line; the other rank exits 0 without work."""
    import socket
    with socket.socket() as sock:
        sock.bind(("127.0.0.1", 0))
        port = sock.getsockname()[1]
    out = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                          "--master-addr", "127.0.0.1", "--master-port", str(port),
                          os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--rows", "50000",
                          "--queries", "4", "--steps", "1", "--warmup", "1", "--cpu-seconds", "0.05"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_selectivity_summary_from_offsets():
    """The bench's achieved-selectivity summary reads answer sizes off the CSR offsets."""
    import importlib.util
    import numpy as np
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    off = np.array([0, 10, 10, 40, 1040], dtype=np.uint64)  # answers of 10, 0, 30, 1000 ids
    s = bench.selectivity_summary(off, 1000)
    assert s["queries"] == 4 and s["empty_queries"] == 1
    assert s["min"] == 0.0 and s["max"] == 1.0 and s["median"] == 0.02
    assert abs(s["mean"] - 1040 / 4000) < 1e-12
    assert bench.selectivity_summary(np.zeros(1, dtype=np.uint64), 1000) == {"queries": 0}


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    return bench


class _PlanTable:
    """Stands in for a table: the plan is the query itself, every zone map in use."""

    def explain(self, q):
        return (any(lo > hi for (_, lo, hi) in q), [] if any(lo > hi for (_, lo, hi) in q) else list(q))

    def zone_map_info(self, j):
        return {"used": True, "mean_width": 0.0}


def _brute_early_break(cols, queries, n, granule, tile=None, max_runs=1024):
    """The same count written out row by row (and tile by tile) with numpy."""
    import numpy as np
    rows = granule // 4
    total = 0
    for q in queries:
        if any(lo > hi for (_, lo, hi) in q):
            continue
        alive = np.ones(n, dtype=bool)
        if tile is not None:
            nt = (n + tile - 1) // tile
            cand = np.ones(nt, dtype=bool)
            for (j, lo, hi) in q:
                for t in range(nt):
                    seg = cols[j][t * tile:(t + 1) * tile]
                    cand[t] &= seg.max() >= lo and seg.min() <= hi
            starts = cand & ~np.concatenate([[False], cand[:-1]])
            if starts.sum() > max_runs:
                idx = np.flatnonzero(cand)
                cand[idx[0]:idx[-1] + 1] = True
            alive = np.repeat(cand, tile)[:n]
        for (j, lo, hi) in q:
            sectors = sum(alive[s:s + rows].any() for s in range(0, n, rows))
            total += granule * sectors
            alive &= (cols[j] >= lo) & (cols[j] <= hi)
        total += 4 * int(alive.sum())
    return total


def test_early_break_byte_count_matches_a_row_by_row_count():
    """bench.py's roofline bytes: sectors that still hold a live row when their column
    is reached, per query in plan order, plus the ids; with tile pruning, only rows of
    candidate tiles are ever live."""
    import numpy as np
    import torch
    bench = _bench_module()
    rng = np.random.default_rng(3)
    n = 9_001
    cols = [np.sort(rng.random(n).astype(np.float32)), rng.random(n).astype(np.float32),
            rng.integers(-5, 5, size=n).astype(np.int32)]
    queries = [[(0, 0.2, 0.4), (1, 0.1, 0.9)], [(2, -1, 1)], [(1, 0.3, 0.31), (2, 0, 4), (0, 0.0, 0.99)],
               [(0, 0.5, 0.4)], [(0, 0.05, 0.06), (2, -5, -5)]]
    dev = [torch.from_numpy(c) for c in cols]
    t = _PlanTable()
    for granule in (32, 64):
        assert bench.early_break_bytes(t, dev, queries, n, granule=granule) == \
            _brute_early_break(cols, queries, n, granule)
        vis = bench.zone_candidates(t, dev, n, tile=512)
        assert bench.early_break_bytes(t, dev, queries, n, granule=granule, visited=vis) == \
            _brute_early_break(cols, queries, n, granule, tile=512)
