"""Parity at the benchmark workloads' full sizes, in the launch configurations bench.py
times: every answer of every query of every workload is compared id for id with the
CPU oracle (Sec. 2.1: the answer set is unique, so count and ids must be identical).

The bulk comparison uses the oracle's dimension-at-a-time evaluation (Sec. 3.2), which
streams each column once; a seeded sample of queries per workload is also answered by
its object-at-a-time evaluation (Sec. 2.2.4). Both are pinned on their own in
tests/test_oracle_pins.py. The other paths the benchmark times (shared scan, prepared
graphs, learned windows, zone maps off, the server) must give the very same ids
(needs a GB300; several minutes, most of it oracle time on the host cores).
"""
import os

import numpy as np
import pytest

import oracle
from paper_1801_03644_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 1
ROW_ORACLE_QUERIES = 8  # per workload, also answered object at a time


@pytest.fixture(scope="module")
def M():
    import torch
    from paper_1801_03644_gb300 import build as B
    B.build()
    from paper_1801_03644_gb300 import mdrq
    mdrq.lib()
    torch.cuda.set_device(0)
    return mdrq


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


def _verify_every_query(M, columns, queries, ids, off, seed):
    """Count and every id of every query against the oracle."""
    nq = len(queries)
    off = np.asarray(off, dtype=np.int64)
    assert off.size == nq + 1 and int(off[0]) == 0 and np.all(np.diff(off) >= 0)
    bad = []
    for q in range(nq):
        a, b = int(off[q]), int(off[q + 1])
        want = oracle.mdrq_columnwise(columns, queries[q], nthreads=NTHREADS)
        if want.size != b - a:
            bad.append(q)
        elif b > a and not np.array_equal(M.as_uint32_numpy(ids[a:b]), want):
            bad.append(q)
    assert not bad, "%d of %d answers differ from the oracle (first: %s)" % (len(bad), nq, bad[:8])
    rng = np.random.default_rng(seed)
    for q in rng.choice(nq, size=min(ROW_ORACLE_QUERIES, nq), replace=False).tolist():
        want = oracle.mdrq(columns, queries[q], nthreads=NTHREADS)
        have = M.as_uint32_numpy(ids[int(off[q]):int(off[q + 1])])
        assert np.array_equal(have, want), q


def _same_answers(ids, off, ids2, off2):
    import torch
    total = int(off[-1])
    return np.array_equal(np.asarray(off), np.asarray(off2)) and bool(torch.equal(ids[:total], ids2[:total]))


def test_uniform_small_full(M):
    """1M x 3, 100 complete-match queries: the batch in one launch, and each query in a
    launch of its own (the cold-cache measurement's configuration)."""
    import torch
    wl = W.uniform_small()
    with M.Table(wl.columns) as t:
        t.set_batch_mode(M.BATCH_PLAIN)
        ids, off = _answer_batch(M, t, wl.queries)
        _verify_every_query(M, wl.columns, wl.queries, ids, off, seed=0)
        for q, query in enumerate(wl.queries):
            one = t.query(query)
            torch.cuda.synchronize()
            assert bool(torch.equal(one, ids[int(off[q]):int(off[q + 1])])), q


def test_mixed_clustered_full(M):
    """1e8 x 8, 1024 partial-match queries: the headline plain batch verified in full;
    the shared scan and the plain batch replayed as a prepared graph identical to it."""
    wl = W.mixed_clustered()
    with M.Table(wl.columns) as t:
        t.set_batch_mode(M.BATCH_PLAIN)
        ids, off = _answer_batch(M, t, wl.queries)
        _verify_every_query(M, wl.columns, wl.queries, ids, off, seed=1)
        with t.prepare(wl.queries) as p:
            ids_g, off_g = p.run()
            assert _same_answers(ids, off, ids_g, off_g)
            del ids_g
        t.set_batch_mode(M.BATCH_SHARED)
        ids2, off2 = _answer_batch(M, t, wl.queries)
        assert _same_answers(ids, off, ids2, off2)


def test_skewed_mixed_types_full(M):
    """5e7 x 32 (float32, Zipf and categorical int32), 256 queries with empty ones."""
    wl = W.skewed_mixed_types()
    with M.Table(wl.columns) as t:
        t.set_batch_mode(M.BATCH_PLAIN)
        ids, off = _answer_batch(M, t, wl.queries)
        _verify_every_query(M, wl.columns, wl.queries, ids, off, seed=2)
        t.set_batch_mode(M.BATCH_SHARED)
        ids2, off2 = _answer_batch(M, t, wl.queries)
        assert _same_answers(ids, off, ids2, off2)


def test_zorder_full(M):
    """2e8 x 4 Z-sorted, 4096 queries: the tile-pruned plain batch verified in full; the
    learned narrower (PLA and MLP) and the scan without zone maps identical to it."""
    wl = W.zorder_learned()
    with M.Table(wl.columns) as t:
        t.set_batch_mode(M.BATCH_PLAIN)
        ids, off = _answer_batch(M, t, wl.queries)
        _verify_every_query(M, wl.columns, wl.queries, ids, off, seed=3)
        for model in (M.MODEL_PLA, M.MODEL_MLP):
            t.learn([0, 1, 2, 3], model, cells=wl.key_bounds)
            t.set_batch_mode(M.BATCH_LEARNED)
            ids2, off2 = _answer_batch(M, t, wl.queries)
            assert _same_answers(ids, off, ids2, off2), model
            del ids2
        t.set_batch_mode(M.BATCH_PLAIN)
        t.set_zone_maps(M.ZONES_OFF)
        ids3, off3 = _answer_batch(M, t, wl.queries)
        assert _same_answers(ids, off, ids3, off3)


def test_serving_table_full(M):
    """2e7 x 16 through the server at its benchmark settings (2 GB result arena, batches
    of up to 512): all 20,000 queries of the stream submitted at once, so that batches
    mix queries of every size; every answer against the oracle."""
    wl = W.serving_table()
    with M.Table(wl.columns) as t:
        srv = M.Server(t, result_bytes=2 << 30, max_batch=512)
        tickets = srv.submit_batch(t.encode_batch(wl.queries))
        bad = []
        for i, tk in enumerate(tickets.tolist()):
            st, ids, cnt, _ = srv.wait(tk)
            assert st == M.OK, i
            got = M.as_uint32_numpy(ids) if ids is not None else np.zeros(0, np.uint32)
            srv.release(tk)
            want = oracle.mdrq_columnwise(wl.columns, wl.queries[i], nthreads=NTHREADS)
            if got.size != cnt or not np.array_equal(got, want):
                bad.append(i)
        assert not bad, "%d of %d served answers differ (first: %s)" % (len(bad), len(tickets), bad[:8])
        rng = np.random.default_rng(4)
        for i in rng.choice(len(wl.queries), size=ROW_ORACLE_QUERIES, replace=False).tolist():
            assert np.array_equal(oracle.mdrq(wl.columns, wl.queries[i], nthreads=NTHREADS),
                                  oracle.mdrq_columnwise(wl.columns, wl.queries[i], nthreads=NTHREADS)), i
        assert srv.stop() == M.OK
