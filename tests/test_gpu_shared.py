"""The batched shared scan (MDRQ_BATCH_SHARED) vs the CPU oracle and vs the plain scan,
id for id (needs a GB300)."""
import numpy as np
import pytest

import oracle
from paper_1801_03644_gb300 import workloads as W
from test_gpu_parity import M, _device, check_batch, edge_queries  # noqa: F401

pytestmark = pytest.mark.gpu

INF = float("inf")


def _variant(name):
    """The shared scan's variants: columns encoded into per-batch codes or searched by
    value, and the row bits kept between the passes or evaluated again."""
    def setup(t):
        t.set_shared_codes(name in ("coded", "coded_no_bits"))
        if name.endswith("no_bits"):
            t.set_shared_bits_budget(0)
    return setup


VARIANTS = pytest.mark.parametrize("variant", ["coded", "values", "coded_no_bits", "values_no_bits"])


@VARIANTS
@pytest.mark.parametrize("n", [1, 31, 32, 33, 4095, 8191, 8192, 8193, 65537, 300_001])
def test_shared_edge_sizes(M, n, variant):
    rng = np.random.default_rng(2000 + n)
    cols = [rng.random(n, dtype=np.float32),
            rng.integers(-40, 40, size=n, dtype=np.int32),
            np.floor(rng.random(n, dtype=np.float32) * 16).astype(np.float32) / 16]
    qs = edge_queries(cols, rng, nrand=40)
    check_batch(M, cols, qs, mode=M.BATCH_SHARED, setup=_variant(variant))


@VARIANTS
def test_shared_special_values(M, variant):
    rng = np.random.default_rng(6)
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
        [(2, 0, 7)], [(2, 8, 100)], [(2, -5, -1)], [(1, 0, -1)], [(0, -0.0, 0.0), (2, 0, 0)],
        [(0, float(np.float32(1e-40)), 1.0)], [(0, -1.0, float(np.float32(-1e-40)))],
    ] * 3
    check_batch(M, cols, qs, mode=M.BATCH_SHARED, setup=_variant(variant))


@VARIANTS
def test_shared_mixed_clustered_many_chunks(M, variant):
    """3M rows x 8 columns, 600 partial-match queries: five chunks of up to 128."""
    wl = W.mixed_clustered(n=3_000_000, nq=600)
    check_batch(M, wl.columns, wl.queries, nthreads=16, mode=M.BATCH_SHARED, setup=_variant(variant))


@VARIANTS
def test_shared_skewed_mixed_types(M, variant):
    """32 columns with int32 Zipf and categorical columns and forced-empty queries."""
    wl = W.skewed_mixed_types(n=2_000_000, nq=256)
    check_batch(M, wl.columns, wl.queries, nthreads=16, mode=M.BATCH_SHARED, setup=_variant(variant))


@VARIANTS
def test_shared_random_pair_queries(M, variant):
    """SYNT-UNI style complete-match random-pair queries (Sec. 7.2.1) on 20 dimensions."""
    wl = W.paper_uniform(n=500_000, d=20, nq=200)
    check_batch(M, wl.columns, wl.queries, nthreads=16, mode=M.BATCH_SHARED, setup=_variant(variant))


def test_shared_coded_and_value_paths_agree_on_a_large_batch(M):
    """2,000 queries over the same columns (16 chunks; up to 4,000 end points in a column's
    union): the coded scan, the value scan and the plain scan give the same ids."""
    import torch
    wl = W.mixed_clustered(n=2_000_003, nq=2000)
    with M.Table(_device(wl.columns)) as t:
        t.set_batch_mode(M.BATCH_PLAIN)
        ids_p, off_p = t.query_batch(wl.queries)
        t.set_batch_mode(M.BATCH_SHARED)
        for coded in (True, False):
            t.set_shared_codes(coded)
            ids_s, off_s = t.query_batch(wl.queries)
            torch.cuda.synchronize()
            assert np.array_equal(off_p, off_s), coded
            assert bool(torch.equal(ids_p, ids_s)), coded
    for q in np.random.default_rng(8).choice(len(wl.queries), size=24, replace=False).tolist():
        assert np.array_equal(M.as_uint32_numpy(ids_p[int(off_p[q]):int(off_p[q + 1])]),
                              oracle.mdrq(wl.columns, wl.queries[q], 16)), q


def test_shared_equals_plain_and_capacity(M):
    import torch
    wl = W.mixed_clustered(n=1_000_003, nq=300)
    cols = _device(wl.columns)
    with M.Table(cols) as t:
        t.set_batch_mode(M.BATCH_PLAIN)
        ids_p, off_p = t.query_batch(wl.queries)
        t.set_batch_mode(M.BATCH_SHARED)
        ids_s, off_s = t.query_batch(wl.queries)
        assert np.array_equal(off_p, off_s)
        assert np.array_equal(M.as_uint32_numpy(ids_p), M.as_uint32_numpy(ids_s))
        # capacity overflow: the prefix below capacity is written, nothing past it
        enc = t.encode_batch(wl.queries)
        total = int(off_s[-1])
        cap = total // 2
        buf = torch.full((cap + 64,), -1, dtype=torch.int32, device="cuda")
        st, off = t.query_batch_raw(enc, buf.data_ptr(), cap, True)
        assert st == M.E_CAPACITY and int(off[-1]) == total
        assert np.array_equal(M.as_uint32_numpy(buf)[:cap], M.as_uint32_numpy(ids_s)[:cap])
        assert np.all(buf[cap:].cpu().numpy() == -1)
        # answers in host memory
        out = np.zeros(total, dtype=np.uint32)
        st, off = t.query_batch_raw(enc, out.ctypes.data, total, False)
        assert st == M.OK and np.array_equal(out, M.as_uint32_numpy(ids_s))
        with pytest.raises(M.MDRQError):
            t.set_batch_mode(7)
