"""mdrq_query_static: the scan entry point that allocates no memory.

Some callers cannot allocate device memory at query time (a serving loop whose device
memory belongs to another allocator's budget, a latency-critical path where
cudaMalloc's implicit synchronisation would stall other streams). For them the library
keeps the scan's scratch in a fixed device array. These tests call that entry point
through the C ABI and check it id for id against the CPU oracle and against the
table-based entry point (mdrq_query), on two calls in a row, since every call reuses
the same scratch array.

This file is named to be collected last, so that a run stopping at the first failure
has already run every other test; it also passes on its own in a fresh process.
"""
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


def test_static_matches_table_entry_point_on_consecutive_calls(M):
    import torch
    wl = W.mixed_clustered(n=1_000_003, nq=12)
    cols = [torch.from_numpy(c).cuda() for c in wl.columns]
    out = torch.full((wl.n,), -1, dtype=torch.int32, device="cuda")
    with M.Table(cols) as t:
        for q in wl.queries:
            want = M.as_uint32_numpy(t.query(q))
            assert np.array_equal(want, oracle.mdrq(wl.columns, q, nthreads=8))
            for _ in range(2):  # the second call finds the first call's scratch contents
                st, cnt = M.query_static(cols, q, out)
                torch.cuda.synchronize()
                assert st == M.OK
                assert cnt == want.size
                assert np.array_equal(M.as_uint32_numpy(out[:cnt]), want)


def test_static_small_and_ragged_sizes(M):
    import torch
    rng = np.random.default_rng(77)
    for n in (1, 5, 4095, 4096, 4097, 70_001):
        x = rng.random(n, dtype=np.float32)
        y = rng.integers(-9, 9, size=n, dtype=np.int32)
        cols = [torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()]
        out = torch.empty(max(1, n), dtype=torch.int32, device="cuda")
        with M.Table(cols) as t:
            for q in ([(0, 0.2, 0.7)], [(0, 0.1, 0.9), (1, -3, 4)], [], [(1, 5, 2)]):
                want = M.as_uint32_numpy(t.query(q))
                assert np.array_equal(want, oracle.mdrq([x, y], q))
                for _ in range(2):
                    st, cnt = M.query_static(cols, q, out)
                    assert st == M.OK and cnt == want.size
                    assert np.array_equal(M.as_uint32_numpy(out[:cnt]), want)


def test_static_allocates_no_device_memory_after_set_up(M):
    import torch
    wl = W.uniform_small(n=2_000_000, nq=3)
    cols = [torch.from_numpy(c).cuda() for c in wl.columns]
    out = torch.empty(wl.n, dtype=torch.int32, device="cuda")
    M.query_static(cols, wl.queries[0], out)  # first call on the device does the set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for q in wl.queries:
        st, _ = M.query_static(cols, q, out)
        assert st == M.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_rejects_sizes_beyond_its_scratch(M):
    import ctypes
    import torch
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    preds = M.encode_query([(0, 0.0, 1.0)], [M.F32])
    cnt = ctypes.c_uint64(123)
    # the length is checked before anything is read
    st = M.lib().mdrq_query_static((ctypes.c_void_p * 1)(x.data_ptr()), (ctypes.c_int32 * 1)(M.F32), 1,
                                   M.STATIC_MAX_ROWS + 1, preds, 1, x.data_ptr(), 16,
                                   ctypes.byref(cnt), None)
    assert st == M.E_INVAL


def test_static_reports_capacity(M):
    import torch
    wl = W.uniform_small(n=300_000, nq=2)
    cols = [torch.from_numpy(c).cuda() for c in wl.columns]
    with M.Table(cols) as t:
        want = M.as_uint32_numpy(t.query(wl.queries[0]))
    assert np.array_equal(want, oracle.mdrq(wl.columns, wl.queries[0]))
    cap = want.size // 2
    out = torch.full((cap + 8,), -1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        st, cnt = M.query_static(cols, wl.queries[0], out[:cap])
        assert st == M.E_CAPACITY and cnt == want.size
        got = M.as_uint32_numpy(out)
        assert np.array_equal(got[:cap], want[:cap])
        assert np.all(out[cap:].cpu().numpy() == -1)
