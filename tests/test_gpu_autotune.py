"""Shared-scan configurations (mdrq_set_shared_config) and the autotuner: every
configuration gives the oracle's answers, and the tuned table still does (needs a GB300)."""
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
def case():
    wl = W.mixed_clustered(n=2_000_003, nq=300)
    want = [oracle.mdrq(wl.columns, q, nthreads=16) for q in wl.queries]
    return wl, want


def _device(cols):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in cols]


def _check(M, t, queries, want):
    import torch
    ids, off = t.query_batch(queries)
    torch.cuda.synchronize()
    got = M.as_uint32_numpy(ids)
    for q, w in enumerate(want):
        assert np.array_equal(got[int(off[q]):int(off[q + 1])], w), q


@pytest.mark.parametrize("keep_bits", [True, False], ids=["bits_kept", "bits_recomputed"])
@pytest.mark.parametrize("unit_rows,image_kib", [(32, 16), (96, 24), (1000, 0), (0, 16), (4096, 208),
                                                 (65536, 40)])
def test_shared_configs_match_oracle(M, case, unit_rows, image_kib, keep_bits):
    """Every shape, with the row bits kept between the passes and recomputed."""
    wl, want = case
    with M.Table(_device(wl.columns)) as t:
        t.set_batch_mode(M.BATCH_SHARED)
        t.set_shared_config(unit_rows, image_kib)
        t.set_shared_bits_budget(2**64 - 1 if keep_bits else 0)
        _check(M, t, wl.queries, want)


def test_config_range_checked(M, case):
    wl, _ = case
    with M.Table(_device(wl.columns[:2])) as t:
        for kib in (8, 15, 209, 1 << 20):
            with pytest.raises(M.MDRQError) as e:
                t.set_shared_config(0, kib)
            assert e.value.status == M.E_INVAL


def test_autotune_then_answers(M, case):
    wl, want = case
    with M.Table(_device(wl.columns)) as t:
        r = t.autotune(wl.queries)
        assert r["mode"] in (M.BATCH_PLAIN, M.BATCH_SHARED)
        assert r["candidates"] >= 5
        assert r["plain_ms"] > 0 and r["shared_default_ms"] > 0
        assert 0 < r["shared_ms"] <= r["shared_default_ms"]
        for mode in (M.BATCH_AUTO, M.BATCH_SHARED, M.BATCH_PLAIN):
            t.set_batch_mode(mode)
            _check(M, t, wl.queries, want)
        # a prepared batch takes the tuned configuration too
        t.set_batch_mode(M.BATCH_AUTO)
        with t.prepare(wl.queries[:64]) as p:
            ids, off = p.run()
            got = M.as_uint32_numpy(ids)
            for q in range(64):
                assert np.array_equal(got[int(off[q]):int(off[q + 1])], want[q])


def test_autotune_without_live_queries(M):
    cols = [np.linspace(0, 1, 5000, dtype=np.float32)]
    with M.Table(_device(cols)) as t:
        r = t.autotune([[(0, 2.0, 3.0)], [(0, 0.9, 0.1)]])
        assert r["candidates"] == 0
