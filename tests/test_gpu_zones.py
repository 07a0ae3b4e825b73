"""Zone maps (mdrq_set_zone_maps): row tiles ruled out by their value ranges are never
visited, and the answers stay those of the oracle on clustered row orders with ragged
tails, duplicated and special values; AUTO picks the clustered columns (needs a GB300)."""
import numpy as np
import pytest

import oracle
from paper_1801_03644_gb300 import workloads as W

pytestmark = pytest.mark.gpu

INF = float("inf")


@pytest.fixture(scope="module")
def M():
    import torch
    from paper_1801_03644_gb300 import build as B
    B.build()
    from paper_1801_03644_gb300 import mdrq
    mdrq.lib()
    torch.cuda.set_device(0)
    return mdrq


def _device(cols):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in cols]


def _check_modes(M, cols, queries, nthreads=8):
    import torch
    want = [oracle.mdrq(cols, q, nthreads=nthreads) for q in queries]
    with M.Table(_device(cols)) as t:
        for zones in (M.ZONES_OFF, M.ZONES_AUTO, M.ZONES_ALL):
            t.set_zone_maps(zones)
            for mode in (M.BATCH_PLAIN, M.BATCH_SHARED):
                t.set_batch_mode(mode)
                ids, off = t.query_batch(queries)
                torch.cuda.synchronize()
                got = M.as_uint32_numpy(ids)
                for q, w in enumerate(want):
                    assert np.array_equal(got[int(off[q]):int(off[q + 1])], w), (zones, mode, q)
            for q, w in enumerate(want[:4]):
                assert np.array_equal(M.as_uint32_numpy(t.query(queries[q])), w)
        t.set_zone_maps(M.ZONES_AUTO)
        info = [t.zone_map_info(j) for j in range(len(cols))]
    return want, info


@pytest.mark.parametrize("n", [1, 127, 128, 129, 4095, 4097, 100_003, 1_000_001])
def test_sorted_and_random_columns(M, n):
    rng = np.random.default_rng(77 + n)
    a = np.sort(rng.random(n, dtype=np.float32))                       # sorted: zones narrow
    b = np.sort(rng.integers(-50, 50, size=n, dtype=np.int32))          # sorted ints, duplicates
    c = rng.random(n, dtype=np.float32)                                 # random: zones wide
    d = np.repeat(rng.integers(0, 5, size=(n + 19_999) // 20_000, dtype=np.int32), 20_000)[:n]  # runs
    cols = [a, b, c, d]
    qs = [[(0, 0.25, 0.5)], [(1, -3, 7)], [(0, 0.1, 0.9), (2, 0.2, 0.4)], [(3, 2, 2)],
          [(1, -50, 49), (3, 0, 4)], [(0, 0.0, 1.0)], [(1, 10, 5)], [(2, 0.5, 0.5000001), (1, 0, 0)],
          [(0, float(a[n // 2]), float(a[n // 2]))], [(3, 1, 3), (0, 0.3, 0.7), (1, -20, 40)]]
    _, info = _check_modes(M, cols, qs)
    if n >= 100_000:
        assert info[0]["used"] and info[1]["used"] and info[3]["used"]
        assert not info[2]["used"] and info[2]["mean_width"] > 0.9


def test_special_float_values(M):
    n = 50_001
    x = np.sort(np.random.default_rng(5).standard_normal(n).astype(np.float32))
    x[:100] = -INF
    x[-100:] = INF
    x[20_000:20_300] = np.float32(-0.0)
    x[20_300:20_700] = np.float32(0.0)
    cols = [x, np.arange(n, dtype=np.int32)]
    qs = [[(0, 0.0, 0.0)], [(0, -0.0, -0.0)], [(0, -INF, -INF)], [(0, INF, INF)], [(0, -INF, 0.0)],
          [(0, 0.0, INF), (1, 1000, 49_000)], [(1, 20_100, 20_650)], [(0, -1.0, 1.0), (1, 0, 127)]]
    _check_modes(M, cols, qs)


def test_zorder_table_learned_and_plain(M):
    """The Z-sorted learned workload at 2M rows: zone maps on, learned and plain answers
    equal the oracle's."""
    import torch
    wl = W.zorder_learned(n=2_000_000, nq=64)
    want = [oracle.mdrq(wl.columns, q, nthreads=16) for q in wl.queries]
    with M.Table(_device(wl.columns)) as t:
        assert all(t.zone_map_info(j)["used"] for j in range(4))
        t.learn([0, 1, 2, 3], M.MODEL_PLA, cells=wl.key_bounds)
        for mode in (M.BATCH_LEARNED, M.BATCH_PLAIN):
            t.set_batch_mode(mode)
            ids, off = t.query_batch(wl.queries)
            torch.cuda.synchronize()
            got = M.as_uint32_numpy(ids)
            for q, w in enumerate(want):
                assert np.array_equal(got[int(off[q]):int(off[q + 1])], w), (mode, q)


def test_zone_mode_checked(M):
    with M.Table(_device([np.zeros(10, np.float32)])) as t:
        with pytest.raises(M.MDRQError):
            t.set_zone_maps(3)
        with pytest.raises(M.MDRQError):
            t.zone_map_info(1)


def test_pruned_tiles_and_run_cap(M):
    """Tile pruning visits fewer tiles on a sorted column; 1024 runs take the exact path,
    1025 runs the one-window fallback; both answer exactly. Also replayed as a graph."""
    import torch
    tiles = 2050
    n = tiles * 4096 - 123
    row = np.arange(n, dtype=np.int64)
    c0 = (((row // 4096) % 2) * 10 + (row % 3)).astype(np.int32)   # alternating tiles
    c1 = row.astype(np.int32)                                      # sorted
    cols = [c0, c1]
    qs = [[(0, 0, 2)],                                  # 1025 runs: fallback window
          [(0, 0, 2), (1, 0, 2048 * 4096 - 1)],         # 1024 runs: exact runs
          [(0, 10, 12), (1, 5000, 5_000_000)],
          [(1, 4096 * 7 + 5, 4096 * 7 + 5)],
          [(0, 3, 9)]]                                  # between the two value bands: no tile qualifies
    want = [oracle.mdrq(cols, q, nthreads=16) for q in qs]
    assert want[4].size == 0
    with M.Table(_device(cols)) as t:
        assert t.zone_map_info(1)["used"]
        t.set_zone_maps(M.ZONES_ALL)
        t.set_batch_mode(M.BATCH_PLAIN)
        for q, w in zip(qs, want):
            assert np.array_equal(M.as_uint32_numpy(t.query(q)), w)
            rows, ntiles = t.zone_scan_info()
            if q is qs[3]:
                assert ntiles == 1 and rows == 4096
            if q is qs[1]:
                assert ntiles == 1024
            if q is qs[4]:
                assert ntiles == 1  # the empty window that closes the answer
        ids, off = t.query_batch(qs)
        torch.cuda.synchronize()
        got = M.as_uint32_numpy(ids)
        for q, w in enumerate(want):
            assert np.array_equal(got[int(off[q]):int(off[q + 1])], w)
        with t.prepare(qs) as p:
            for _ in range(2):
                ids, off = p.run()
                got = M.as_uint32_numpy(ids)
                for q, w in enumerate(want):
                    assert np.array_equal(got[int(off[q]):int(off[q + 1])], w)
