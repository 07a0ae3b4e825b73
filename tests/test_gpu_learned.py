"""The learned range narrower (MDRQ_BATCH_LEARNED) vs the CPU oracle and the plain scan,
id for id, with both models (needs a GB300)."""
import numpy as np
import pytest

import oracle
from paper_1801_03644_gb300 import workloads as W
from test_gpu_parity import M, _device  # noqa: F401

pytestmark = pytest.mark.gpu


def _learned_answers(M, cols_np, queries, model, dims=(0, 1, 2, 3), cells=None):
    import torch
    cols = _device(cols_np)
    with M.Table(cols) as t:
        info = t.learn(list(dims), model, cells=cells)
        t.set_batch_mode(M.BATCH_LEARNED)
        ids, off = t.query_batch(queries)
        torch.cuda.synchronize()
        got = M.as_uint32_numpy(ids).copy()
        t.set_batch_mode(M.BATCH_PLAIN)
        ids_p, off_p = t.query_batch(queries)
        plain = M.as_uint32_numpy(ids_p).copy()
    return info, got, off, plain, off_p


MODELS = pytest.mark.parametrize("model", [1, 2, 3], ids=["pla", "mlp", "none"])


@MODELS
def test_learned_matches_oracle_and_plain(M, model):
    wl = W.zorder_learned(n=2_000_003, nq=160)
    info, got, off, plain, off_p = _learned_answers(M, wl.columns, wl.queries, model, cells=wl.key_bounds)
    if model == 3:
        assert info["max_error"] == wl.n and info["segments"] == 0
    else:
        # the two-stage MLP-rooted model stays within a small multiple of the PLA's
        # error (about 0.02% of n on this table); its network alone misses by ~20% of n
        assert info["max_error"] < (0.001 if model == 1 else 0.005) * wl.n, info
    assert np.array_equal(off, off_p) and np.array_equal(got, plain)
    for q, query in enumerate(wl.queries):
        want = oracle.mdrq(wl.columns, query, nthreads=8)
        assert np.array_equal(got[int(off[q]):int(off[q + 1])], want), q


@MODELS
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
    info, got, off, plain, off_p = _learned_answers(M, wl.columns, qs, model, cells=wl.key_bounds)
    assert np.array_equal(off, off_p) and np.array_equal(got, plain)
    for q, query in enumerate(qs):
        want = oracle.mdrq(wl.columns, query, nthreads=8)
        assert np.array_equal(got[int(off[q]):int(off[q + 1])], want), (q, query)


@pytest.mark.parametrize("n", [1, 5, 4096, 4097, 70_001])
def test_learned_small_tables(M, n):
    wl = W.zorder_learned(n=n, nq=24)
    info, got, off, plain, off_p = _learned_answers(M, wl.columns, wl.queries, 1, cells=wl.key_bounds)
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


@MODELS
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


# ---------------------------------------------------------------- the model's error, off the GPU

def _pla_predict(exp, keys):
    """A PLA's prediction for every key, in the arithmetic the model states: the last
    knot at or below the key (knot 0 below the first), the key offset rounded to
    float32, times the float32 slope, added in double to the knot's row."""
    S = exp["segments"]
    kk = exp["knot_key"].astype(np.int64)
    seg = np.clip(np.searchsorted(kk[:S], keys, side="right") - 1, 0, S - 1)
    k0 = kk[seg]
    dk = np.where(keys >= k0, (keys - k0).astype(np.float32), -((k0 - keys).astype(np.float32)))
    prod = (dk * exp["slope"][seg]).astype(np.float32)
    return exp["knot_pos"][seg].astype(np.float64) + prod.astype(np.float64)


def _fma32(a, b, c):
    """float32 fused multiply-add: the float32 product is exact in float64, and the sum
    is rounded once more to float32 (a double rounding that can differ from a true FMA
    in the last bit, rarely)."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def _mlp_predict(exp, keys):
    """The two-stage model's prediction: network output -> leaf -> the leaf's line."""
    w = exp["mlp"]
    H = 32
    W1, b1, W2 = w[0:H], w[H:2 * H], w[2 * H:2 * H + H * H].reshape(H, H)
    b2, W3, b3 = w[2 * H + H * H:3 * H + H * H], w[3 * H + H * H:4 * H + H * H], w[4 * H + H * H]
    kmin = exp["key_min"]
    d = np.where(keys >= kmin, (keys - kmin).astype(np.float32), -((kmin - keys).astype(np.float32)))
    u = (d * exp["key_inv"]).astype(np.float32)
    h1 = [np.maximum(np.float32(0), _fma32(np.full_like(u, W1[i]), u, np.full_like(u, b1[i]))) for i in range(H)]
    h2 = []
    for o in range(H):
        a = np.full_like(u, b2[o])
        for i in range(H):
            a = _fma32(np.full_like(u, W2[o, i]), h1[i], a)
        h2.append(np.maximum(np.float32(0), a))
    y = np.full_like(u, b3)
    for i in range(H):
        y = _fma32(np.full_like(u, W3[i]), h2[i], y)
    L = exp["segments"]
    y = (y * np.float32(L)).astype(np.float32)
    leaf = np.where(y > 0, np.minimum(np.floor(np.where(y > 0, y, 0)), L - 1), 0).astype(np.int64)
    kk = exp["knot_key"].astype(np.int64)
    k0 = kk[leaf]
    dk = np.where(keys >= k0, (keys - k0).astype(np.float32), -((k0 - keys).astype(np.float32)))
    prod = (dk * exp["slope"][leaf]).astype(np.float32)
    return exp["knot_pos"][leaf].astype(np.float64) + prod.astype(np.float64)


@pytest.mark.parametrize("model", [1, 2], ids=["pla", "mlp"])
def test_max_error_recomputed_from_the_parameters(M, model):
    """mdrq_learn_info's error is the largest |prediction - row| over every key of the
    table: recomputed here on the CPU from the exported parameters, exhaustively."""
    wl = W.zorder_learned(n=1_000_003, nq=4)
    keys = W.zorder_key(wl.columns, wl.key_bounds).astype(np.int64)
    assert np.all(np.diff(keys) >= 0)
    with M.Table(_device(wl.columns)) as t:
        info = t.learn([0, 1, 2, 3], model, cells=wl.key_bounds)
        exp = t.learn_export()
    assert exp["kind"] == model and exp["max_error"] == info["max_error"]
    pred = _pla_predict(exp, keys) if model == 1 else _mlp_predict(exp, keys)
    err = int(np.ceil(np.abs(pred - np.arange(wl.n, dtype=np.float64))).max())
    if model == 1:
        assert err == info["max_error"]
    else:
        # a last-bit difference can move a key near a leaf boundary to the next leaf
        assert abs(err - info["max_error"]) <= 2 + 0.05 * info["max_error"], (err, info["max_error"])


def test_models_search_fewer_keys_than_no_model(M):
    """With the same key ranges, a model's window leaves its binary searches fewer keys
    to read than a search over the whole key column (mdrq_learn_search_info)."""
    import torch
    wl = W.zorder_learned(n=2_000_003, nq=64)
    with M.Table(_device(wl.columns)) as t:
        t.set_batch_mode(M.BATCH_LEARNED)
        probes = {}
        for model in (1, 2, 3):
            t.learn([0, 1, 2, 3], model, cells=wl.key_bounds)
            t.query_batch(wl.queries)
            torch.cuda.synchronize()
            probes[model] = t.learn_search_info()
    ranges = {m: r for m, (r, _) in probes.items()}
    assert ranges[1] == ranges[2] == ranges[3] > 0
    assert probes[1][1] < probes[3][1] and probes[2][1] < probes[3][1], probes


def test_equal_width_and_quantile_cells_both_exact(M):
    """The same rows sorted by the equal-width key and by the quantile-cell key: each
    table learned with its own cells answers exactly; a table learned with cells it is
    not sorted by is refused; bad cell bounds are refused."""
    import ctypes
    wl = W.zorder_learned(n=400_003, nq=48)
    for sort_cells in (None, wl.key_bounds):
        key = W.zorder_key(wl.columns, sort_cells)
        o = np.argsort(key, kind="stable")
        cols = [c[o] for c in wl.columns]
        info, got, off, plain, off_p = _learned_answers(M, cols, wl.queries, 1, cells=sort_cells)
        assert np.array_equal(off, off_p) and np.array_equal(got, plain)
        for q, query in enumerate(wl.queries):
            assert np.array_equal(got[int(off[q]):int(off[q + 1])], oracle.mdrq(cols, query, 4)), q
    with M.Table(_device(wl.columns)) as t:  # sorted by the quantile key, not the equal-width one
        with pytest.raises(M.MDRQError) as e:
            t.learn([0, 1, 2, 3], 1)
        assert e.value.status == M.E_INVAL
        bad = np.array(wl.key_bounds[0][::-1])  # descending
        assert M.lib().mdrq_set_key_cells(t.handle, 0, bad.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                          255) == M.E_INVAL
        assert M.lib().mdrq_set_key_cells(t.handle, 0, None, 7) == M.E_INVAL
        assert M.lib().mdrq_set_key_cells(t.handle, 9, None, 0) == M.E_INVAL
