"""The continuous-batching server (mdrq_server_*): every answer in the mix equals the
query's answer alone (CPU oracle and the table's own mdrq_query), id for id; admission
by result memory defers queries without losing any (needs a GB300)."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_1801_03644_gb300 import workloads as W
from test_gpu_parity import M, _device  # noqa: F401

pytestmark = pytest.mark.gpu


def _run_stream(M, server, queries, rate, release=True):
    """Submit on a Poisson schedule from this thread; a second thread waits, copies the
    answers to the host and releases them. Returns {index: (status, ids, latency)}."""
    arrivals = W.poisson_arrivals(rate, len(queries))
    tickets = [None] * len(queries)
    got = {}
    done = threading.Event()

    def consumer():
        i = 0
        while i < len(queries):
            while tickets[i] is None:
                time.sleep(0.0001)
            st, ids, cnt, lat = server.wait(tickets[i])
            got[i] = (st, M.as_uint32_numpy(ids) if ids is not None else np.zeros(0, np.uint32), cnt, lat)
            if release and st == M.OK:
                server.release(tickets[i])
            i += 1
        done.set()

    th = threading.Thread(target=consumer)
    th.start()
    t0 = time.perf_counter()
    for i, q in enumerate(queries):
        wait = arrivals[i] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        tickets[i] = server.submit(q)
    th.join(timeout=300)
    assert done.is_set()
    return got


def test_answers_alone_equal_answers_in_the_mix(M):
    wl = W.serving_table(n=1_000_003, nq=400)
    cols = _device(wl.columns)
    with M.Table(cols) as t:
        alone = [M.as_uint32_numpy(t.query(q)).copy() for q in wl.queries]
        srv = M.Server(t, result_bytes=256 << 20, max_batch=64)
        got = _run_stream(M, srv, wl.queries, rate=20_000)
        stats = srv.stats()
        assert srv.stop() == M.OK
    for i, q in enumerate(wl.queries):
        st, ids, cnt, lat = got[i]
        assert st == M.OK and cnt == ids.size
        assert np.array_equal(ids, alone[i]), i
        assert np.array_equal(ids, oracle.mdrq(wl.columns, q, 8)), i
        assert lat > 0
    assert stats["completed"] == len(wl.queries)
    assert stats["batches"] >= 2 and 0 < stats["p50_us"] <= stats["p99_us"]


def test_admission_by_result_memory(M):
    """An arena that holds only a few answers: queries wait for memory, in order, and
    every answer is still exact; an answer larger than the arena fails cleanly."""
    wl = W.serving_table(n=500_000, nq=120)
    cols = _device(wl.columns)
    with M.Table(cols) as t:
        sizes = [t.query(q).numel() for q in wl.queries]
        biggest = max(sizes)
        arena = max(4 * biggest + 16, sum(sizes) * 4 // 10)
        srv = M.Server(t, result_bytes=arena, max_batch=32)
        got = _run_stream(M, srv, wl.queries, rate=50_000)
        stats = srv.stats()
        assert stats["deferred"] > 0
        # a query whose answer cannot fit at all
        small = M.Server(t, result_bytes=4 * max(1, biggest // 2), max_batch=8)
        i_big = int(np.argmax(sizes))
        tk = small.submit(wl.queries[i_big])
        st, ids, cnt, lat = small.wait(tk)
        assert st == M.E_CAPACITY and cnt == biggest
        assert small.stop() == M.OK
        assert srv.stop() == M.OK
    for i, q in enumerate(wl.queries):
        st, ids, cnt, lat = got[i]
        assert st == M.OK
        assert np.array_equal(ids, oracle.mdrq(wl.columns, q, 8)), i


def test_stop_answers_queued_queries(M):
    wl = W.serving_table(n=200_000, nq=50)
    cols = _device(wl.columns)
    with M.Table(cols) as t:
        srv = M.Server(t, result_bytes=64 << 20, max_batch=16)
        tickets = [srv.submit(q) for q in wl.queries]
        res = [srv.wait(tk) for tk in tickets]
        assert all(r[0] == M.OK for r in res)
        for (st, ids, cnt, lat), q in zip(res, wl.queries):
            got = M.as_uint32_numpy(ids) if ids is not None else np.zeros(0, np.uint32)
            assert np.array_equal(got, oracle.mdrq(wl.columns, q, 4))
        assert srv.stop() == M.OK


def test_small_batches_and_bursts(M):
    """A slow stream (batches of one or two: the plain-scan path) and a burst (large
    batches: the shared scan) on the same server; every answer exact."""
    wl = W.serving_table(n=700_001, nq=120)
    cols = _device(wl.columns)
    with M.Table(cols) as t:
        srv = M.Server(t, result_bytes=256 << 20, max_batch=64)
        slow = _run_stream(M, srv, wl.queries[:30], rate=400)
        burst = [srv.submit(q) for q in wl.queries[30:]]
        res = []
        for tk in burst:  # copied to the host while the server (and its arena) lives
            st, ids, cnt, lat = srv.wait(tk)
            res.append((st, M.as_uint32_numpy(ids).copy() if ids is not None else np.zeros(0, np.uint32)))
        stats = srv.stats()
        assert srv.stop() == M.OK
    for i in range(30):
        st, ids, cnt, lat = slow[i]
        assert st == M.OK and np.array_equal(ids, oracle.mdrq(wl.columns, wl.queries[i], 8)), i
    for j, (st, got) in enumerate(res):
        assert st == M.OK and np.array_equal(got, oracle.mdrq(wl.columns, wl.queries[30 + j], 8)), j
    assert stats["batches"] >= 20


def test_bulk_submit_and_wait_many(M):
    """mdrq_server_submit_batch / mdrq_server_wait_many: the same answers (sizes) as one
    query at a time, answers released by the wait; a bad query submits nothing."""
    wl = W.serving_table(n=400_003, nq=300)
    cols = _device(wl.columns)
    with M.Table(cols) as t:
        sizes = [t.query(q).numel() for q in wl.queries]
        srv = M.Server(t, result_bytes=64 << 20, max_batch=64)
        enc = t.encode_batch(wl.queries)
        tk = srv.submit_batch(enc)
        assert tk.size == len(wl.queries) and np.all(np.diff(tk.astype(np.int64)) == 1)
        status, counts, lat = srv.wait_many(tk[:150], release=True)
        assert np.all(status == M.OK) and np.array_equal(counts, np.asarray(sizes[:150], np.uint64))
        assert np.all(lat > 0)
        # the rest: waited without release, then read one by one
        status, counts, lat = srv.wait_many(tk[150:], release=False)
        assert np.all(status == M.OK)
        for k, q in zip(tk[150:160], wl.queries[150:160]):
            st, ids, cnt, _ = srv.wait(int(k))
            got = M.as_uint32_numpy(ids).copy() if ids is not None else np.zeros(0, np.uint32)
            assert np.array_equal(got, oracle.mdrq(wl.columns, q, 8))
        with pytest.raises(M.MDRQError):
            srv.wait_many(tk[:1])  # already released
        assert srv.stop() == M.OK


def test_allocation_failure_ends_the_batch_and_the_queue(M):
    """A batch whose scratch allocation fails (injected on the host, before any of its
    GPU work) ends with MDRQ_E_NOMEM, and so does every query queued behind it; submit
    then refuses with that status, and stop returns it. No GPU fault is involved."""
    wl = W.serving_table(n=200_000, nq=600)
    with M.Table(_device(wl.columns)) as t:
        srv = M.Server(t, result_bytes=1 << 26, max_batch=64)
        t.inject_fault(M.FAULT_NOMEM)
        tickets = srv.submit_batch(t.encode_batch(wl.queries))
        status, counts, _ = srv.wait_many(tickets, release=False, timeout_us=30_000_000)
        failed = status == M.E_NOMEM
        # queries proven empty on the host are answered at submit, before any batch
        answered_at_submit = (status == M.OK) & (counts == 0)
        assert np.all(failed | answered_at_submit), np.unique(status)
        assert failed.sum() >= 64 and failed.sum() > 64  # the failed batch and the queue behind it
        with pytest.raises(M.MDRQError) as e:
            srv.submit(wl.queries[0])
        assert e.value.status == M.E_NOMEM
        assert srv.stop() == M.E_NOMEM
    # the table itself stays usable
    with M.Table(_device(wl.columns)) as t:
        assert np.array_equal(M.as_uint32_numpy(t.query(wl.queries[0])), oracle.mdrq(wl.columns, wl.queries[0]))
