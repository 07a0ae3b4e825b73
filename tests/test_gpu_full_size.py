"""Parity at the benchmark workloads' full sizes, in the launch configurations bench.py
times: every query's answer is checked for order and range, a sample of queries against
the CPU oracle id for id, and for every query a sample of rows both ways (a row is in
the answer iff it satisfies the query) (needs a GB300; a few minutes)."""
import numpy as np
import pytest

import oracle
from paper_1801_03644_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ORACLE_QUERIES = 8   # answered in full by the oracle per workload
ROW_SAMPLES = 64     # rows checked both ways per query


@pytest.fixture(scope="module")
def M():
    import torch
    from paper_1801_03644_gb300 import build as B
    B.build()
    from paper_1801_03644_gb300 import mdrq
    mdrq.lib()
    torch.cuda.set_device(0)
    return mdrq


def _predicate_rows(columns, query, rows):
    """Which of ``rows`` satisfy the query: the closed-interval test of Sec. 2.1 in the
    columns' own types (numpy, independent of both the kernels and the oracle)."""
    ok = np.ones(rows.size, dtype=bool)
    for dim, lo, hi in query:
        x = columns[dim][rows]
        lo_t = np.asarray(lo, dtype=x.dtype)
        hi_t = np.asarray(hi, dtype=x.dtype)
        ok &= (lo_t <= x) & (x <= hi_t)
    return ok


def _answer_batch(M, t, queries):
    """The bench's call: one mdrq_query_batch into an exactly sized device buffer."""
    import torch
    enc = t.encode_batch(queries)
    probe = torch.empty(1, dtype=torch.int32, device="cuda")
    st, off = t.query_batch_raw(enc, probe.data_ptr(), 0, True)
    assert st in (M.OK, M.E_CAPACITY)
    ids = torch.empty(max(1, int(off[-1])), dtype=torch.int32, device="cuda")
    st, off = t.query_batch_raw(enc, ids.data_ptr(), ids.numel(), True)
    assert st == M.OK
    torch.cuda.synchronize()
    return ids, off


def _check(M, columns, queries, ids, off, seed, oracle_queries=ORACLE_QUERIES):
    import torch
    n = columns[0].size
    nq = len(queries)
    assert int(off[0]) == 0 and np.all(np.diff(off.astype(np.int64)) >= 0)
    total = int(off[-1])
    dev = ids[:total]  # int32: every id is below 2^31
    # every id in range and strictly ascending inside its query's segment
    assert total == 0 or (int(dev.min()) >= 0 and int(dev.max()) < n)
    if total > 1:
        inc = dev[1:] > dev[:-1]
        starts = torch.zeros(total, dtype=torch.bool, device=dev.device)
        o = torch.from_numpy(off[1:-1].astype(np.int64)).to(dev.device)  # positions
        o = o[(o > 0) & (o < total)]
        starts[o] = True
        assert bool(torch.all(inc | starts[1:]))
    rng = np.random.default_rng(seed)
    # sampled rows, both ways, for every query
    for q in range(nq):
        rows = np.unique(rng.integers(0, n, size=ROW_SAMPLES))
        a, b = int(off[q]), int(off[q + 1])
        seg = dev[a:b]
        rt = torch.from_numpy(rows.astype(np.int32)).to(dev.device)
        if b > a:
            pos = torch.searchsorted(seg, rt).clamp(max=b - a - 1)
            member = (seg[pos] == rt).cpu().numpy()
        else:
            member = np.zeros(rows.size, dtype=bool)
        want = _predicate_rows(columns, queries[q], rows)
        assert np.array_equal(member, want), q
        # and a few of the query's own ids satisfy it
        if b > a:
            pick = rng.integers(a, b, size=min(16, b - a))
            mine = ids[torch.from_numpy(pick).to(dev.device)].cpu().numpy().astype(np.int64)
            assert np.all(_predicate_rows(columns, queries[q], mine)), q
    # whole answers of a sample of queries against the oracle
    for q in rng.choice(nq, size=min(oracle_queries, nq), replace=False):
        want = oracle.mdrq(columns, queries[int(q)], nthreads=16)
        have = M.as_uint32_numpy(ids[int(off[q]):int(off[q + 1])])
        assert have.size == want.size and np.array_equal(have, want), int(q)


def test_mixed_clustered_full(M):
    """1e8 x 8, 1024 partial-match queries: the headline plain batch, and the shared
    scan's answers identical to it."""
    import torch
    wl = W.mixed_clustered()
    with M.Table(wl.columns) as t:
        t.set_batch_mode(M.BATCH_PLAIN)
        ids, off = _answer_batch(M, t, wl.queries)
        _check(M, wl.columns, wl.queries, ids, off, seed=1)
        t.set_batch_mode(M.BATCH_SHARED)
        ids2, off2 = _answer_batch(M, t, wl.queries)
        assert np.array_equal(off, off2)
        assert bool(torch.equal(ids[: int(off[-1])], ids2[: int(off2[-1])]))


def test_skewed_mixed_types_full(M):
    """5e7 x 32 (float32, Zipf and categorical int32), 256 queries with empty ones."""
    wl = W.skewed_mixed_types()
    with M.Table(wl.columns) as t:
        t.set_batch_mode(M.BATCH_PLAIN)
        ids, off = _answer_batch(M, t, wl.queries)
        _check(M, wl.columns, wl.queries, ids, off, seed=2)


def test_zorder_full(M):
    """2e8 x 4 Z-sorted, 4096 queries: tile-pruned plain batch checked, and the learned
    narrower (PLA) and the scan without zone maps identical to it."""
    import torch
    wl = W.zorder_learned()
    with M.Table(wl.columns) as t:
        t.set_batch_mode(M.BATCH_PLAIN)
        ids, off = _answer_batch(M, t, wl.queries)
        _check(M, wl.columns, wl.queries, ids, off, seed=3)
        total = int(off[-1])
        t.learn([0, 1, 2, 3], M.MODEL_PLA)
        t.set_batch_mode(M.BATCH_LEARNED)
        ids2, off2 = _answer_batch(M, t, wl.queries)
        assert np.array_equal(off, off2) and bool(torch.equal(ids[:total], ids2[:total]))
        del ids2
        t.set_batch_mode(M.BATCH_PLAIN)
        t.set_zone_maps(M.ZONES_OFF)
        ids3, off3 = _answer_batch(M, t, wl.queries)
        assert np.array_equal(off, off3) and bool(torch.equal(ids[:total], ids3[:total]))
        del ids3


def test_serving_table_full(M):
    """2e7 x 16 through the server at its benchmark batch size: sampled answers exact."""
    wl = W.serving_table()
    qs = wl.queries[:3000]
    with M.Table(wl.columns) as t:
        srv = M.Server(t, result_bytes=2 << 30, max_batch=512)
        tickets = [srv.submit(q) for q in qs]
        rng = np.random.default_rng(4)
        check = set(rng.choice(len(qs), size=ORACLE_QUERIES, replace=False).tolist())
        for i, tk in enumerate(tickets):
            st, ids, cnt, lat = srv.wait(tk)
            assert st == M.OK
            got = M.as_uint32_numpy(ids).copy() if ids is not None else np.zeros(0, np.uint32)
            srv.release(tk)
            assert got.size == cnt and (got.size < 2 or np.all(np.diff(got.astype(np.int64)) > 0))
            rows = np.unique(rng.integers(0, wl.n, size=ROW_SAMPLES))
            pos = np.minimum(np.searchsorted(got, rows), max(0, got.size - 1))
            member = (got[pos] == rows) if got.size else np.zeros(rows.size, dtype=bool)
            assert np.array_equal(member, _predicate_rows(wl.columns, qs[i], rows)), i
            if i in check:
                assert np.array_equal(got, oracle.mdrq(wl.columns, qs[i], nthreads=16)), i
        assert srv.stop() == M.OK
