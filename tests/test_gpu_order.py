"""Output orders of the scan (mdrq_set_output_order): look-back and staged give the
oracle's answers id for id, on ragged sizes, skewed and mixed-type tables, short answer
buffers (tiles that miss the staging buffer are recomputed), host answers split over
several launches, prepared batches, single queries, and the windowed launches of tile
pruning and the learned narrower (needs a GB300)."""
import numpy as np
import pytest

import oracle
from paper_1801_03644_gb300 import workloads as W
from test_gpu_parity import SIZES, _device, check_batch, edge_queries

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    from paper_1801_03644_gb300 import build as B
    B.build()
    from paper_1801_03644_gb300 import mdrq
    mdrq.lib()
    torch.cuda.set_device(0)
    return mdrq


def order(M, mode):
    return lambda t: t.set_output_order(mode)


ORDERS = pytest.mark.parametrize("order_mode", [1, 2], ids=["lookback", "staged"])


@pytest.mark.parametrize("n", SIZES)
def test_edge_sizes_staged(M, n):
    rng = np.random.default_rng(3000 + n)
    cols = [rng.random(n, dtype=np.float32),
            rng.integers(-40, 40, size=n, dtype=np.int32),
            np.floor(rng.random(n, dtype=np.float32) * 16).astype(np.float32) / 16]
    check_batch(M, cols, edge_queries(cols, rng), mode=M.BATCH_PLAIN, setup=order(M, M.ORDER_STAGED))


@ORDERS
def test_mixed_clustered_orders(M, order_mode):
    wl = W.mixed_clustered(n=3_000_000, nq=96)
    check_batch(M, wl.columns, wl.queries, nthreads=16, mode=M.BATCH_PLAIN, setup=order(M, order_mode))


@ORDERS
def test_skewed_mixed_types_orders(M, order_mode):
    wl = W.skewed_mixed_types(n=2_000_000, nq=256)
    check_batch(M, wl.columns, wl.queries, nthreads=16, mode=M.BATCH_PLAIN, setup=order(M, order_mode))


def test_uniform_1M_staged_and_auto_agree(M):
    """The 1M x 3 batch of 100 queries is staged under ORDER_AUTO; forced look-back and
    forced staged give the oracle's answers too."""
    wl = W.uniform_small()
    for mode in (M.ORDER_AUTO, M.ORDER_LOOKBACK, M.ORDER_STAGED):
        check_batch(M, wl.columns, wl.queries, mode=M.BATCH_PLAIN, setup=order(M, mode))


@pytest.mark.parametrize("frac", [0.0, 0.01, 0.34, 0.99])
def test_short_buffer_staged_keeps_the_prefix(M, frac):
    """A staged batch whose answer overflows the caller's buffer: the staging buffer has the
    caller's capacity, so later tiles miss it and the ordering pass recomputes those that
    land below capacity. Every id below capacity is the oracle's; nothing past it is
    written; the reported total is exact."""
    import torch
    wl = W.mixed_clustered(n=1_000_003, nq=40)
    cols = _device(wl.columns)
    want = [oracle.mdrq(wl.columns, q, 16) for q in wl.queries]
    cat = np.concatenate(want)
    total = cat.size
    cap = int(total * frac)
    with M.Table(cols) as t:
        t.set_batch_mode(M.BATCH_PLAIN)
        t.set_output_order(M.ORDER_STAGED)
        enc = t.encode_batch(wl.queries)
        buf = torch.full((cap + 256,), -1, dtype=torch.int32, device="cuda")
        st, off = t.query_batch_raw(enc, buf.data_ptr(), cap, True)
        assert st == M.E_CAPACITY and int(off[-1]) == total
        assert np.array_equal(np.diff(off.astype(np.int64)), [w.size for w in want])
        got = M.as_uint32_numpy(buf)
        assert np.array_equal(got[:cap], cat[:cap])
        assert np.all(buf[cap:].cpu().numpy() == -1)


def test_host_answers_over_several_launches_staged(M):
    """Pageable host answers split the batch into several launches (each later launch's
    output starts where the previous one ended); every launch is staged."""
    wl = W.mixed_clustered(n=12_000_017, nq=24)
    with M.Table(_device(wl.columns)) as t:
        t.set_batch_mode(M.BATCH_PLAIN)
        t.set_output_order(M.ORDER_STAGED)
        want = [oracle.mdrq(wl.columns, q, 16) for q in wl.queries]
        cat = np.concatenate(want)
        enc = t.encode_batch(wl.queries)
        out = np.full(cat.size + 7, 0xFFFFFFFF, dtype=np.uint32)
        st, off = t.query_batch_raw(enc, out.ctypes.data, cat.size, False)
        assert st == M.OK
        assert t.last_scan_stats()[0] > 1  # launches
        assert np.array_equal(out[:cat.size], cat) and np.all(out[cat.size:] == 0xFFFFFFFF)
        assert np.array_equal(np.diff(off.astype(np.int64)), [w.size for w in want])


def test_prepared_batch_staged(M):
    """A prepared (graph-captured) plain batch with staged output, replayed twice."""
    import torch
    wl = W.uniform_small(n=400_009, nq=64)
    want = [oracle.mdrq(wl.columns, q, 8) for q in wl.queries]
    cat = np.concatenate(want)
    with M.Table(_device(wl.columns)) as t:
        t.set_batch_mode(M.BATCH_PLAIN)
        t.set_output_order(M.ORDER_STAGED)
        out = torch.full((cat.size + 16,), -1, dtype=torch.int32, device="cuda")
        with t.prepare(wl.queries, out=out) as p:
            for _ in range(2):
                out.fill_(-1)
                ids, off = p.run()
                torch.cuda.synchronize()
                assert np.array_equal(M.as_uint32_numpy(out)[:cat.size], cat)
                assert np.array_equal(np.diff(np.asarray(off, dtype=np.int64)), [w.size for w in want])


def test_single_query_staged(M):
    import torch
    rng = np.random.default_rng(11)
    n = 3_000_001
    cols = [rng.random(n, dtype=np.float32), rng.random(n, dtype=np.float32)]
    q = [(0, 0.2, 0.6), (1, 0.1, 0.15)]
    want = oracle.mdrq(cols, q, 8)
    with M.Table(_device(cols)) as t:
        for mode in (M.ORDER_LOOKBACK, M.ORDER_STAGED):
            t.set_output_order(mode)
            out = torch.empty(want.size, dtype=torch.int32, device="cuda")
            assert np.array_equal(M.as_uint32_numpy(t.query(q, out=out)), want)


@ORDERS
@pytest.mark.parametrize("batch", ["zones", "learned_pla", "learned_none"])
def test_windowed_orders(M, order_mode, batch):
    """Windowed launches (tile pruning on the Z-sorted table; the learned narrower's
    windows): look-back and staged answers equal the oracle's."""
    import torch
    wl = W.zorder_learned(n=2_000_003, nq=96)
    want = [oracle.mdrq(wl.columns, q, nthreads=16) for q in wl.queries]
    with M.Table(_device(wl.columns)) as t:
        t.set_output_order(order_mode)
        if batch == "zones":
            t.set_zone_maps(M.ZONES_ALL)
            t.set_batch_mode(M.BATCH_PLAIN)
        else:
            t.learn([0, 1, 2, 3], M.MODEL_PLA if batch == "learned_pla" else M.MODEL_NONE, cells=wl.key_bounds)
            t.set_batch_mode(M.BATCH_LEARNED)
        ids, off = t.query_batch(wl.queries)
        torch.cuda.synchronize()
        got = M.as_uint32_numpy(ids)
        for q, w in enumerate(want):
            assert np.array_equal(got[int(off[q]):int(off[q + 1])], w), (batch, q)


@pytest.mark.parametrize("batch", ["zones", "learned"])
def test_windowed_short_buffer_staged(M, batch):
    """A staged windowed batch into a buffer of a third of its answer: the prefix is the
    oracle's, nothing past capacity is written, the total is exact."""
    import torch
    wl = W.zorder_learned(n=1_000_003, nq=48)
    cat = np.concatenate([oracle.mdrq(wl.columns, q, nthreads=16) for q in wl.queries])
    cap = cat.size // 3
    with M.Table(_device(wl.columns)) as t:
        t.set_output_order(M.ORDER_STAGED)
        if batch == "zones":
            t.set_zone_maps(M.ZONES_ALL)
            t.set_batch_mode(M.BATCH_PLAIN)
        else:
            t.learn([0, 1, 2, 3], M.MODEL_PLA, cells=wl.key_bounds)
            t.set_batch_mode(M.BATCH_LEARNED)
        enc = t.encode_batch(wl.queries)
        buf = torch.full((cap + 256,), -1, dtype=torch.int32, device="cuda")
        st, off = t.query_batch_raw(enc, buf.data_ptr(), cap, True)
        assert st == M.E_CAPACITY and int(off[-1]) == cat.size
        got = M.as_uint32_numpy(buf)
        assert np.array_equal(got[:cap], cat[:cap])
        assert np.all(buf[cap:].cpu().numpy() == -1)


def test_staging_unavailable_falls_back_to_lookback(M):
    """A staged launch whose staging buffers cannot be had (a host-side fault: the
    allocation reported as failed) orders its output by look-back instead: one kernel
    instead of the scan and the three ordering kernels, the same answers."""
    import torch
    wl = W.mixed_clustered(n=1_000_003, nq=40)
    want = [oracle.mdrq(wl.columns, q, 16) for q in wl.queries]
    with M.Table(_device(wl.columns)) as t:
        t.set_batch_mode(M.BATCH_PLAIN)
        t.set_output_order(M.ORDER_STAGED)
        t.scan_timing(True)
        for fault, kernels_per_scan in ((True, 1), (False, 4)):
            t.scan_timing_read(reset=True)
            if fault:
                t.inject_fault(M.FAULT_STAGE_NOMEM)
            out = torch.empty(sum(w.size for w in want), dtype=torch.int32, device="cuda")
            ids, off = t.query_batch(wl.queries, out=out)  # one call: the buffer fits
            torch.cuda.synchronize()
            tm = t.scan_timing_read(reset=True)
            assert tm["scan_launches"] >= 1
            assert tm["kernel_launches"] == kernels_per_scan * tm["scan_launches"], (fault, tm)
            got = M.as_uint32_numpy(ids)
            for q, w in enumerate(want):
                assert np.array_equal(got[int(off[q]):int(off[q + 1])], w), (fault, q)
        t.scan_timing(False)


def test_bad_order_mode_rejected(M):
    wl = W.uniform_small(n=1000, nq=1)
    with M.Table(wl.columns) as t:
        with pytest.raises(M.MDRQError):
            t.set_output_order(7)
