"""The learned range narrower (MDRQ_BATCH_LEARNED) vs the CPU oracle and the plain scan,
id for id, with both models (needs a GB300)."""
import numpy as np
import pytest

import oracle
from paper_1801_03644_gb300 import workloads as W
from test_gpu_parity import M, _device  # noqa: F401

pytestmark = pytest.mark.gpu


def _learned_answers(M, cols_np, queries, model, dims=(0, 1, 2, 3)):
    import torch
    cols = _device(cols_np)
    with M.Table(cols) as t:
        info = t.learn(list(dims), model)
        t.set_batch_mode(M.BATCH_LEARNED)
        ids, off = t.query_batch(queries)
        torch.cuda.synchronize()
        got = M.as_uint32_numpy(ids).copy()
        t.set_batch_mode(M.BATCH_PLAIN)
        ids_p, off_p = t.query_batch(queries)
        plain = M.as_uint32_numpy(ids_p).copy()
    return info, got, off, plain, off_p


@pytest.mark.parametrize("model", [1, 2], ids=["pla", "mlp"])
def test_learned_matches_oracle_and_plain(M, model):
    wl = W.zorder_learned(n=2_000_003, nq=160)
    info, got, off, plain, off_p = _learned_answers(M, wl.columns, wl.queries, model)
    assert info["max_error"] < wl.n
    assert np.array_equal(off, off_p) and np.array_equal(got, plain)
    for q, query in enumerate(wl.queries):
        want = oracle.mdrq(wl.columns, query, nthreads=8)
        assert np.array_equal(got[int(off[q]):int(off[q + 1])], want), q


@pytest.mark.parametrize("model", [1, 2], ids=["pla", "mlp"])
def test_learned_partial_and_odd_queries(M, model):
    wl = W.zorder_learned(n=300_001, nq=40)
    rng = np.random.default_rng(9)
    qs = []
    for q in wl.queries[:20]:
        keep = sorted(rng.choice(4, size=int(rng.integers(1, 4)), replace=False).tolist())
        qs.append([p for p in q if p[0] in keep])  # partial-match on the key dims
    qs += [[], [(0, -1.0, 2.0)], [(1, 0.5, 0.25)], [(2, 0.999, 5.0), (3, -3.0, 0.001)],
           [(0, 0.0, 0.0)], [(3, 0.3, 0.3)], [(0, 0.1, 0.9), (0, 0.2, 0.3)]]
    r = int(rng.integers(0, wl.n))
    qs.append([(j, float(wl.columns[j][r]), float(wl.columns[j][r])) for j in range(4)])
    info, got, off, plain, off_p = _learned_answers(M, wl.columns, qs, model)
    assert np.array_equal(off, off_p) and np.array_equal(got, plain)
    for q, query in enumerate(qs):
        want = oracle.mdrq(wl.columns, query, nthreads=8)
        assert np.array_equal(got[int(off[q]):int(off[q + 1])], want), (q, query)


@pytest.mark.parametrize("n", [1, 5, 4096, 4097, 70_001])
def test_learned_small_tables(M, n):
    wl = W.zorder_learned(n=n, nq=24)
    info, got, off, plain, off_p = _learned_answers(M, wl.columns, wl.queries, 1)
    assert np.array_equal(off, off_p) and np.array_equal(got, plain)
    for q, query in enumerate(wl.queries):
        assert np.array_equal(got[int(off[q]):int(off[q + 1])], oracle.mdrq(wl.columns, query, 2))


def test_learned_on_key_subset_with_extra_column(M):
    """The key over 2 of 3 columns; the third column is only filtered by the scan."""
    rng = np.random.default_rng(10)
    n = 500_000
    a, b, c = (rng.random(n, dtype=np.float32) for _ in range(3))
    key = W.zorder_key([a, b])
    o = np.argsort(key, kind="stable")
    cols = [a[o], b[o], c[o]]
    qs = [[(0, 0.1, 0.3), (1, 0.2, 0.25), (2, 0.0, 0.5)], [(2, 0.4, 0.6)], [(0, 0.5, 0.51)]] * 4
    info, got, off, plain, off_p = _learned_answers(M, cols, qs, 1, dims=(0, 1))
    assert np.array_equal(got, plain) and np.array_equal(off, off_p)


def test_learn_rejects_unsorted_rows_and_missing_model(M):
    rng = np.random.default_rng(11)
    cols = _device([rng.random(10_000, dtype=np.float32) for _ in range(2)])
    with M.Table(cols) as t:
        with pytest.raises(M.MDRQError) as e:
            t.learn([0, 1], 1)
        assert e.value.status == M.E_INVAL
        t.set_batch_mode(M.BATCH_LEARNED)
        with pytest.raises(M.MDRQError) as e:
            t.query_batch([[(0, 0.1, 0.2)]])
        assert e.value.status == M.E_INVAL
    icol = _device([np.arange(100, dtype=np.int32)])
    with M.Table(icol) as t:
        with pytest.raises(M.MDRQError):
            t.learn([0], 1)  # key dimensions must be float32


@pytest.mark.parametrize("model", [1, 2], ids=["pla", "mlp"])
@pytest.mark.parametrize("dims", [(1,), (2, 0), (0, 2, 1), (3, 1, 0, 2)], ids=["1d", "2d", "3d", "4d_permuted"])
def test_learned_key_widths_and_orders(M, model, dims):
    """Keys over 1 to 4 of the columns, in any column order (the table sorted by that
    key), with boxes inside, across and outside the unit cube; answers equal the
    oracle's and the plain scan's."""
    rng = np.random.default_rng(100 + len(dims))
    n = 300_007
    cols = [rng.random(n, dtype=np.float32) for _ in range(4)]
    cols[3] = (cols[3] ** 3).astype(np.float32)  # a skewed column
    key = W.zorder_key([cols[j] for j in dims])
    o = np.argsort(key, kind="stable")
    cols = [c[o] for c in cols]
    qs = []
    for k in range(64):
        q = []
        for j in range(4):
            if rng.random() < 0.7:
                lo = float(rng.uniform(-0.1, 1.0))
                hi = lo + float(rng.uniform(0.0, 0.5))
                q.append((j, lo, hi))
        qs.append(q)
    qs += [[(dims[0], 0.5, 0.5)], [(dims[0], 1.2, 2.0)], [(dims[0], -1.0, -0.5)], [(dims[-1], 0.0, 0.99999994)]]
    info, got, off, plain, off_p = _learned_answers(M, cols, qs, model, dims=dims)
    assert np.array_equal(off, off_p) and np.array_equal(got, plain)
    for q, query in enumerate(qs):
        assert np.array_equal(got[int(off[q]):int(off[q + 1])], oracle.mdrq(cols, query, 4)), q
