"""GPU scan vs the CPU oracle, id for id, through the C ABI (needs a GB300)."""
import math

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


def check_batch(M, columns, queries, on_device=True, nthreads=8, mode=None, setup=None):
    """Every query's answer equals the oracle's (count and every id). ``setup(table)``
    may configure the table first."""
    import torch
    cols = _device(columns) if on_device else columns
    with M.Table(cols) as t:
        if mode is not None:
            t.set_batch_mode(mode)
        if setup is not None:
            setup(t)
        ids, off = t.query_batch(queries)
        torch.cuda.synchronize()
        got = M.as_uint32_numpy(ids)
    assert off[0] == 0 and np.all(np.diff(off.astype(np.int64)) >= 0)
    for q, query in enumerate(queries):
        want = oracle.mdrq(columns, query, nthreads=nthreads)
        have = got[int(off[q]):int(off[q + 1])]
        assert have.size == want.size, (q, query, have.size, want.size)
        assert np.array_equal(have, want), (q, query)
    return off


def edge_queries(columns, rng, nrand=6):
    d = len(columns)
    n = columns[0].size
    qs = [[], [(0, 0.5, 0.25)] if columns[0].dtype == np.float32 else [(0, 5, 4)]]
    full = []
    for j, c in enumerate(columns):
        full.append((j, -INF, INF) if c.dtype == np.float32 else (j, -2**31, 2**31 - 1))
    qs.append(full)
    for _ in range(nrand):
        q = []
        for j in sorted(rng.choice(d, size=int(rng.integers(1, d + 1)), replace=False).tolist()):
            c = columns[j]
            if n:
                a, b = c[rng.integers(0, n)], c[rng.integers(0, n)]
            else:
                a, b = 0, 1
            lo, hi = (a, b) if a <= b else (b, a)
            q.append((j, lo.item() if hasattr(lo, "item") else lo, hi.item() if hasattr(hi, "item") else hi))
        qs.append(q)
    if n:
        r = int(rng.integers(0, n))
        qs.append([(j, columns[j][r].item(), columns[j][r].item()) for j in range(d)])
    return qs


SIZES = [0, 1, 2, 3, 4, 5, 31, 32, 33, 127, 128, 129, 511, 512, 513, 1023, 1024, 1025,
         2047, 2048, 2049, 4095, 4096, 4097, 8191, 65537, 300_001]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("on_device", [True, False], ids=["device_cols", "host_cols"])
@pytest.mark.parametrize("mode", [1, 2], ids=["plain", "shared"])
def test_edge_sizes(M, n, on_device, mode):
    rng = np.random.default_rng(1000 + n)
    cols = [rng.random(n, dtype=np.float32),
            rng.integers(-40, 40, size=n, dtype=np.int32),
            np.floor(rng.random(n, dtype=np.float32) * 16).astype(np.float32) / 16]
    check_batch(M, cols, edge_queries(cols, rng), on_device=on_device, mode=mode)


@pytest.mark.parametrize("mode", [1, 2], ids=["plain", "shared"])
def test_mixed_types_and_special_values(M, mode):
    rng = np.random.default_rng(5)
    n = 70_001
    x = rng.standard_normal(n).astype(np.float32)
    x[::97] = np.float32(-0.0)
    x[::89] = np.float32(0.0)
    x[5] = np.float32(INF)
    x[6] = np.float32(-INF)
    i = rng.integers(-2**31, 2**31 - 1, size=n, dtype=np.int64).astype(np.int32)
    i[7] = -2**31
    i[8] = 2**31 - 1
    cols = [x, i, rng.integers(0, 8, size=n, dtype=np.int32)]
    qs = [
        [(0, 0.0, 0.0)], [(0, -0.0, -0.0)], [(0, INF, INF)], [(0, -INF, -INF)],
        [(0, -INF, 0.0), (1, 0, 2**31 - 1)], [(1, -2**31, -2**31)], [(1, 2**31 - 1, 2**31 - 1)],
        [(2, 3, 3), (2, 2, 5)], [(2, 3, 5), (2, 6, 7)], [(0, -1.0, 1.0), (0, -0.5, 2.0), (2, 1, 6)],
        [(2, 0, 7)], [(2, 8, 100)], [(2, -5, -1)], [(1, 0, -1)],
    ]
    check_batch(M, cols, qs, mode=mode)


MODES = pytest.mark.parametrize("mode", [1, 2], ids=["plain", "shared"])


def test_shared_hints_on_wide_and_integer_columns(M):
    """The shared scan's bucket hints on columns whose ranges stress the float bucket
    function: int32 over the whole range, floats spanning 1e-30 .. 1e30 and tiny ranges
    near 1.0, with many queries so that hints are built; plain and shared agree with the
    oracle."""
    rng = np.random.default_rng(77)
    n = 200_003
    wide_i = rng.integers(-2**31, 2**31 - 1, size=n, dtype=np.int64).astype(np.int32)
    wide_i[:3] = [-2**31, 2**31 - 1, 0]
    wide_f = (10.0 ** rng.uniform(-30, 30, size=n) * rng.choice([-1, 1], size=n)).astype(np.float32)
    narrow_f = (1.0 + rng.integers(0, 200, size=n) * np.float32(2 ** -23)).astype(np.float32)
    cols = [wide_i, wide_f, narrow_f]
    qs = []
    for k in range(300):
        a, b = sorted(rng.choice(n, size=2, replace=False))
        c0 = np.sort(wide_i[[a, b]])
        c1 = np.sort(wide_f[[a, b]])
        c2 = np.sort(narrow_f[[a, b]])
        pick = k % 4
        q = []
        if pick in (0, 3):
            q.append((0, int(c0[0]), int(c0[1])))
        if pick in (1, 3):
            q.append((1, float(c1[0]), float(c1[1])))
        if pick in (2, 3):
            q.append((2, float(c2[0]), float(c2[1])))
        qs.append(q)
    check_batch(M, cols, qs, mode=1)
    check_batch(M, cols, qs, mode=2)


@MODES
def test_uniform_1M_all_queries(M, mode):
    """1M x 3 uniform, 100 complete-match queries of about 1% selectivity."""
    wl = W.uniform_small()
    off = check_batch(M, wl.columns, wl.queries, mode=mode)
    assert abs(off[-1] / 100 - 10_000) < 3 * math.sqrt(1e4) / 10 * 3


@MODES
def test_mixed_clustered_reduced(M, mode):
    """The 8-column uniform + cluster-mixture recipe at 3M rows, 96 partial-match queries."""
    wl = W.mixed_clustered(n=3_000_000, nq=96)
    check_batch(M, wl.columns, wl.queries, nthreads=16, mode=mode)


@MODES
def test_mixed_clustered_large_tiles(M, mode):
    """12M rows: the 4096-row tile variant, several hundred tiles per SM wave."""
    wl = W.mixed_clustered(n=12_000_017, nq=24)
    check_batch(M, wl.columns, wl.queries, nthreads=16, mode=mode)


@MODES
def test_skewed_mixed_types_reduced(M, mode):
    """32 columns (float32 uniform, int32 Zipf, int32 categorical), 256 queries including
    empty ones, at 2M rows."""
    wl = W.skewed_mixed_types(n=2_000_000, nq=256)
    off = check_batch(M, wl.columns, wl.queries, nthreads=16, mode=mode)
    assert np.sum(np.diff(off.astype(np.int64)) == 0) >= 5


def test_single_query_paths(M):
    """mdrq_query with device and host answers, and the exact-capacity edge."""
    import torch
    wl = W.mixed_clustered(n=500_000, nq=6)
    cols = _device(wl.columns)
    with M.Table(cols) as t:
        for q in wl.queries:
            want = oracle.mdrq(wl.columns, q, 8)
            dev = M.as_uint32_numpy(t.query(q))
            host = t.query_host(q)
            assert np.array_equal(dev, want) and np.array_equal(host, want)
            if want.size:
                exact = torch.empty(want.size, dtype=torch.int32, device="cuda")
                assert np.array_equal(M.as_uint32_numpy(t.query(q, out=exact)), want)


def test_capacity_overflow_reports_required_size(M):
    import torch
    wl = W.uniform_small(n=200_000, nq=8)
    cols = _device(wl.columns)
    want = [oracle.mdrq(wl.columns, q, 8) for q in wl.queries]
    total = sum(w.size for w in want)
    cat = np.concatenate(want)
    with M.Table(cols) as t:
        t.set_batch_mode(M.BATCH_PLAIN)
        enc = t.encode_batch(wl.queries)
        cap = total // 3
        buf = torch.full((cap + 64,), -1, dtype=torch.int32, device="cuda")
        st, off = t.query_batch_raw(enc, buf.data_ptr(), cap, True)
        assert st == M.E_CAPACITY and int(off[-1]) == total
        got = M.as_uint32_numpy(buf)
        assert np.array_equal(got[:cap], cat[:cap])
        assert np.all(buf[cap:].cpu().numpy() == -1)  # nothing past capacity
        # host answers with too small a buffer
        st, off = t.query_batch_raw(enc, np.zeros(1, np.uint32).ctypes.data, 0, False)
        assert st == M.E_CAPACITY and int(off[-1]) == total


def test_host_answer_batch(M):
    wl = W.uniform_small(n=100_003, nq=10)
    with M.Table(wl.columns) as t:
        enc = t.encode_batch(wl.queries)
        want = [oracle.mdrq(wl.columns, q, 4) for q in wl.queries]
        total = sum(w.size for w in want)
        out = np.zeros(total, dtype=np.uint32)
        st, off = t.query_batch_raw(enc, out.ctypes.data, total, False)
        assert st == M.OK
        assert np.array_equal(out, np.concatenate(want))


def test_nan_rejected(M):
    x = np.linspace(0, 1, 1000, dtype=np.float32)
    x[500] = np.nan
    with pytest.raises(M.MDRQError) as e:
        M.Table(_device([x]))
    assert e.value.status == M.E_NAN
    y = np.linspace(0, 1, 1000, dtype=np.float32)
    with M.Table(_device([y])) as t:
        with pytest.raises(M.MDRQError) as e:
            t.query([(0, float("nan"), 1.0)])
        assert e.value.status == M.E_INVAL
        with pytest.raises(ValueError):
            t.query([(3, 0.0, 1.0)])


def test_misaligned_device_column_rejected(M):
    import torch
    x = torch.zeros(1001, dtype=torch.float32, device="cuda")
    with pytest.raises(M.MDRQError) as e:
        M.Table([x[1:]])
    assert e.value.status == M.E_INVAL


def test_repeat_calls_reuse_scratch(M):
    """Hundreds of launches on one table (tile-state epochs, claim counter) stay exact."""
    wl = W.uniform_small(n=250_000, nq=300)
    check_batch(M, wl.columns, wl.queries, mode=1)


@pytest.mark.parametrize("host", [1, 0, 2], ids=["staged", "auto", "direct"])
@pytest.mark.parametrize("mode", [1, 2], ids=["plain", "shared"])
def test_host_answers_pinned_and_pageable(M, mode, host):
    """Host answers: staged (a plain batch's launches copied out one by one while the
    next runs; the batch scans more than 2 GiB of columns, so it is split into several
    launches) or written by the kernels themselves into page-locked memory (direct).
    Auto takes the staged copies here, since the plain batch's output is staged
    (mdrq_set_output_order AUTO: 64 queries of 733 tiles). The result and the capacity
    rule are those of the device path, for a page-locked and a pageable buffer, with the
    capacity cut inside the batch."""
    import torch
    wl = W.mixed_clustered(n=3_000_017, nq=64)
    want = [oracle.mdrq(wl.columns, q, 8) for q in wl.queries]
    cat = np.concatenate(want)
    total = cat.size
    with M.Table(_device(wl.columns)) as t:
        t.set_batch_mode(mode)
        t.set_host_answers(host)
        enc = t.encode_batch(wl.queries)
        pinned = torch.full((total + 64,), -1, dtype=torch.int32, pin_memory=True)
        st, off = t.query_batch_raw(enc, pinned.data_ptr(), total, False)
        assert st == M.OK and int(off[-1]) == total
        if mode == 1:
            launches, scanned = t.last_scan_stats()
            assert scanned >= 2 << 30
            assert (launches >= 2) if host in (0, 1) else (launches == 1), launches
        got = pinned.numpy().view(np.uint32)
        assert np.array_equal(got[:total], cat)
        assert np.all(pinned.numpy()[total:] == -1)
        # too small: the first `cap` ids, nothing beyond
        pinned.fill_(-1)
        cap = total // 3
        st, off = t.query_batch_raw(enc, pinned.data_ptr(), cap, False)
        assert st == M.E_CAPACITY and int(off[-1]) == total
        assert np.array_equal(pinned.numpy().view(np.uint32)[:cap], cat[:cap])
        assert np.all(pinned.numpy()[cap:] == -1)
        # pageable host memory: staged, except in direct mode, which refuses it
        page = np.zeros(total, dtype=np.uint32)
        st, off = t.query_batch_raw(enc, page.ctypes.data, total, False)
        if host == 2:
            assert st == M.E_INVAL
        else:
            assert st == M.OK and np.array_equal(page, cat)
        # a single query into page-locked memory
        one = np.zeros(0, dtype=np.uint32)
        if want[0].size:
            pin1 = torch.full((want[0].size,), -1, dtype=torch.int32, pin_memory=True)
            cnt = M.ctypes.c_uint64(0)
            preds = M.encode_query(wl.queries[0], t.dtypes)
            st = M.lib().mdrq_query(t.handle, preds, len(wl.queries[0]), pin1.data_ptr(), pin1.numel(),
                                    M.ctypes.byref(cnt), 0, None)
            one = pin1.numpy().view(np.uint32)
            assert st == M.OK and cnt.value == want[0].size
        assert np.array_equal(one, want[0])


def test_explain_query_plan(M):
    """mdrq_explain_query: repeated dimensions are intersected, predicates every value
    satisfies are dropped, queries no value can meet are answered empty, and the rest
    are evaluated most selective first; the answer follows the plan."""
    rng = np.random.default_rng(5)
    n = 100_000
    x = rng.random(n, dtype=np.float32)
    y = rng.integers(-5, 6, size=n, dtype=np.int32)
    with M.Table(_device([x, y])) as t:
        assert t.explain([(0, 0.2, 0.5), (1, -100, 100)]) == (False, [(0, float(np.float32(0.2)),
                                                                          float(np.float32(0.5)))])
        assert t.explain([(0, 0.2, 0.5), (0, 0.3, 0.9)]) == (False, [(0, float(np.float32(0.3)),
                                                                         float(np.float32(0.5)))])
        assert t.explain([(0, 0.5, 0.2)]) == (True, [])
        assert t.explain([(1, 10, 20)]) == (True, [])
        assert t.explain([]) == (False, [])
        empty, plan = t.explain([(0, 0.0, 0.9), (1, 0, 0)])
        assert not empty and [p[0] for p in plan] == [1, 0]  # y = 0 holds for 1 in 11 rows
        for q in ([(0, 0.2, 0.5), (1, -100, 100)], [(0, 0.0, 0.9), (1, 0, 0)]):
            _, plan = t.explain(q)
            assert np.array_equal(M.as_uint32_numpy(t.query(q)), oracle.mdrq([x, y], plan))
