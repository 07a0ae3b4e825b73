"""Prepared batches (mdrq_prepare_batch): the batch recorded as a CUDA graph and
replayed; every replay's answer equals the CPU oracle's, id for id (needs a GB300)."""
import numpy as np
import pytest

import oracle
from paper_1801_03644_gb300 import workloads as W

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


@pytest.fixture(scope="module")
def mixed():
    wl = W.mixed_clustered(n=3_000_000, nq=64)
    want = [oracle.mdrq(wl.columns, q, nthreads=16) for q in wl.queries]
    return wl, want


def _device(cols):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in cols]


def _check(M, ids, off, want):
    got = M.as_uint32_numpy(ids)
    assert int(off[0]) == 0 and int(off[-1]) == sum(w.size for w in want)
    for q, w in enumerate(want):
        assert np.array_equal(got[int(off[q]):int(off[q + 1])], w), q


@pytest.mark.parametrize("mode", [0, 1, 2], ids=["auto", "plain", "shared"])
def test_replays_match_oracle(M, mixed, mode):
    import torch
    wl, want = mixed
    with M.Table(_device(wl.columns)) as t:
        t.set_batch_mode(mode)
        with t.prepare(wl.queries) as p:
            _check(M, p.out, p.first_offsets, want)
            assert p.kernels() >= 1
            for _ in range(3):
                p.out.fill_(-1)
                ids, off = p.run()
                torch.cuda.synchronize()
                _check(M, ids, off, want)


def test_replays_back_to_back_and_interleaved_with_table_calls(M, mixed):
    """Several replays queued on one stream, and plain table calls (own scratch) between
    replays, leave every answer exact."""
    import torch
    wl, want = mixed
    with M.Table(_device(wl.columns)) as t:
        t.set_batch_mode(M.BATCH_PLAIN)
        with t.prepare(wl.queries) as p:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                for _ in range(5):
                    p.launch(s)
                off = p.wait(s)
            _check(M, p.out[: int(off[-1])], off, want)
            for k in range(3):
                q = wl.queries[k]
                dev = M.as_uint32_numpy(t.query(q))  # the table's own scratch and tags
                assert np.array_equal(dev, want[k])
                ids, off = p.run()
                _check(M, ids, off, want)
                # a batch call on the table between replays
                ids2, off2 = t.query_batch(wl.queries[10:18])
                torch.cuda.synchronize()
                _check(M, ids2, off2, want[10:18])


def test_uniform_small_plain_replays(M):
    wl = W.uniform_small()
    want = [oracle.mdrq(wl.columns, q, nthreads=8) for q in wl.queries]
    with M.Table(_device(wl.columns)) as t:
        with t.prepare(wl.queries) as p:
            for _ in range(2):
                ids, off = p.run()
                _check(M, ids, off, want)


def test_empty_and_degenerate_batches(M):
    import torch
    rng = np.random.default_rng(3)
    cols = [rng.random(10_001, dtype=np.float32), rng.integers(0, 9, 10_001, dtype=np.int32)]
    qs = [[(0, 0.7, 0.2)], [(1, 20, 30)], [], [(1, 3, 3), (0, 0.25, 0.75)]]
    want = [oracle.mdrq(cols, q, 4) for q in qs]
    with M.Table(_device(cols)) as t:
        with t.prepare(qs) as p:
            ids, off = p.run()
            _check(M, ids, off, want)
        with t.prepare([]) as p:
            ids, off = p.run()
            assert off.tolist() == [0]
        with t.prepare([[(0, 2.0, 3.0)]]) as p:  # proven empty on the host
            ids, off = p.run()
            assert off.tolist() == [0, 0]


def test_capacity_and_learned_mode_rejected(M, mixed):
    import torch
    wl, want = mixed
    total = sum(w.size for w in want)
    with M.Table(_device(wl.columns)) as t:
        small = torch.empty(max(1, total // 2), dtype=torch.int32, device="cuda")
        with pytest.raises(M.MDRQError) as e:
            t.prepare(wl.queries, out=small)
        assert e.value.status == M.E_CAPACITY
        t.set_batch_mode(M.BATCH_LEARNED)
        with pytest.raises(M.MDRQError) as e:
            t.prepare(wl.queries[:2])
        assert e.value.status == M.E_INVAL
