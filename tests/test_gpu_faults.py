"""Failure detection without a GPU fault: a bounded device wait that runs out is
reported as MDRQ_E_TIMEOUT and leaves the table usable; an injected allocation
failure is reported as MDRQ_E_NOMEM. Nothing here traps, faults or hangs the GPU:
the wait that is made to run out is bounded (about a second) by construction."""
import time

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


def test_lookback_wait_runs_out_and_table_recovers(M):
    import torch
    wl = W.uniform_small(n=100_000, nq=3)
    cols = [torch.from_numpy(c).cuda() for c in wl.columns]
    with M.Table(cols) as t:
        q = wl.queries[0]
        want = oracle.mdrq(wl.columns, q, 4)
        t.inject_fault(M.FAULT_SKIP_TILES, 3)
        t0 = time.time()
        with pytest.raises(M.MDRQError) as e:
            t.query(q)
        assert e.value.status == M.E_TIMEOUT
        assert time.time() - t0 < 30
        # the context and the table still work, and answer exactly
        for q in wl.queries:
            assert np.array_equal(M.as_uint32_numpy(t.query(q)), oracle.mdrq(wl.columns, q, 4))
        assert np.array_equal(M.as_uint32_numpy(t.query(wl.queries[0])), want)


def test_injected_allocation_failure(M):
    import torch
    wl = W.uniform_small(n=50_000, nq=2)
    cols = [torch.from_numpy(c).cuda() for c in wl.columns]
    with M.Table(cols) as t:
        t.inject_fault(M.FAULT_NOMEM)
        with pytest.raises(M.MDRQError) as e:
            t.query(wl.queries[0])
        assert e.value.status == M.E_NOMEM
        got = M.as_uint32_numpy(t.query(wl.queries[1]))
        assert np.array_equal(got, oracle.mdrq(wl.columns, wl.queries[1], 4))
        with pytest.raises(M.MDRQError):
            t.inject_fault(99)
