"""The seeded input generators: shapes, ranges and selectivity statistics (no GPU)."""
import math

import numpy as np

import oracle
from paper_1801_03644_gb300 import workloads as W


def test_uniform_small_shape_and_mean_count():
    """1M x 3 uniform, 100 queries of width 0.01^(1/3): each count is binomial with
    mean 10,000 (sd 99.5), so the mean of 100 counts lies within 10,000 +- 3*9.95."""
    wl = W.uniform_small()
    assert wl.n == 1_000_000 and wl.d == 3 and len(wl.queries) == 100
    for c in wl.columns:
        assert c.dtype == np.float32 and c.min() >= 0.0 and c.max() < 1.0
    # the table is default_rng(0).random((3, n), float32)
    ref = np.random.default_rng(0).random((3, 1_000_000), dtype=np.float32)
    assert all(np.array_equal(a, b) for a, b in zip(wl.columns, ref))
    counts = []
    for q in wl.queries:
        assert [p[0] for p in q] == [0, 1, 2]
        for (_, lo, hi) in q:
            assert 0.0 <= lo <= hi < 1.0
            assert abs((hi - lo) - W.UNIFORM_SMALL_WIDTH) < 1e-6
        counts.append(len(oracle.mdrq(wl.columns, q, nthreads=8)))
    sd = math.sqrt(1e6 * 0.01 * 0.99)
    assert abs(np.mean(counts) - 10_000) < 3 * sd / math.sqrt(100)


def test_mixed_clustered_small_scale():
    wl = W.mixed_clustered(n=200_000, nq=64)
    assert wl.d == 8 and len(wl.queries) == 64
    for c in wl.columns:
        assert c.dtype == np.float32 and c.min() >= 0.0 and c.max() < 1.0
    # dims 4-7 share one cluster id per row: 20 joint clusters of sigma 0.02 fill few
    # of the 10^4 cells of a 10-per-axis grid, where uniform dims fill nearly all
    def cells_for_99pct(cols):
        cell = np.zeros(wl.n, dtype=np.int64)
        for c in cols:
            cell = cell * 10 + np.minimum((c * 10).astype(np.int64), 9)
        cnt = np.sort(np.bincount(cell, minlength=10 ** 4))[::-1]
        return int(np.searchsorted(np.cumsum(cnt), 0.99 * wl.n)) + 1
    assert cells_for_99pct(wl.columns[4:8]) < 1500
    assert cells_for_99pct(wl.columns[0:4]) > 9000
    for q in wl.queries:
        dims = [p[0] for p in q]
        assert 2 <= len(dims) <= 8 and dims == sorted(set(dims))
        for (_, lo, hi) in q:
            assert lo <= hi


def test_independent_uniform_dims_multiply():
    """Sec. 2.1: for independent dimensions sel = prod_j sel_j."""
    wl = W.mixed_clustered(n=400_000, nq=200)
    n = wl.n
    checked = 0
    for q in wl.queries:
        if any(p[0] >= 4 for p in q) or len(q) < 2:
            continue
        sel = len(oracle.mdrq(wl.columns, q, 8)) / n
        prod = 1.0
        for p in q:
            prod *= len(oracle.mdrq(wl.columns, [p], 8)) / n
        if prod * n > 400:
            assert abs(sel - prod) < 5 * math.sqrt(prod / n) + 1e-4, (q, sel, prod)
            checked += 1
    assert checked >= 3


def test_skewed_mixed_types_small_scale():
    wl = W.skewed_mixed_types(n=100_000, nq=128)
    assert wl.d == 32
    assert all(c.dtype == np.float32 for c in wl.columns[:16])
    assert all(c.dtype == np.int32 for c in wl.columns[16:])
    z = wl.columns[16]
    assert z.min() >= 1 and z.max() <= 1_000_000
    # Zipf(1.2): P(1) = 1 / zeta_{1e6}(1.2) ~ 0.18
    assert 0.15 < np.mean(z == 1) < 0.21
    cat = wl.columns[24]
    assert cat.min() == 0 and cat.max() == 63
    empties = sum(1 for q in wl.queries if len(oracle.mdrq(wl.columns, q, 8)) == 0)
    assert empties >= 3
    for q in wl.queries:
        assert 3 <= len(q) <= 12


def test_generators_are_deterministic():
    a = W.mixed_clustered(n=10_000, nq=8)
    b = W.mixed_clustered(n=10_000, nq=8)
    assert all(np.array_equal(x, y) for x, y in zip(a.columns, b.columns))
    assert a.queries == b.queries


def _deinterleave(key: np.ndarray, j: int) -> np.ndarray:
    """Cell of dimension j read back out of a Morton key: bit 4b + j of the key is bit
    b of the cell (the inverse of the interleave, computed bit by bit per row)."""
    out = np.zeros(key.shape[0], dtype=np.uint32)
    for b in range(8):
        out |= ((key >> np.uint32(4 * b + j)) & np.uint32(1)) << np.uint32(b)
    return out


def test_zorder_key_interleaves_cells():
    rng = np.random.default_rng(3)
    cols = [rng.random(5000, dtype=np.float32) for _ in range(4)]
    cols[0][:3] = [0.0, np.float32(W.ONE_BELOW), 0.5]
    key = W.zorder_key(cols)
    for j in range(4):
        want = np.minimum(np.floor(cols[j].astype(np.float64) * 256.0), 255).astype(np.uint32)
        assert np.array_equal(_deinterleave(key, j), want)
    assert list(_deinterleave(key[:3], 0)) == [0, 255, 128]
    # a single row: dimension 0 in the lowest bit of each nibble
    one = W.zorder_key([np.array([1.0 / 256], np.float32), np.zeros(1, np.float32),
                        np.zeros(1, np.float32), np.array([3.0 / 256], np.float32)])
    assert int(one[0]) == (1 << 0) | (1 << 3) | (1 << 7)


def test_zorder_table_is_sorted_and_normalised():
    wl = W.zorder_learned(n=60_000, nq=16)
    assert wl.d == 4 and all(c.dtype == np.float32 for c in wl.columns)
    key = W.zorder_key(wl.columns, wl.key_bounds)
    assert np.all(key[1:] >= key[:-1])  # rows in key order
    for c in wl.columns:
        assert c.min() >= 0.0 and c.max() <= W.ONE_BELOW
    for j in (1, 3):  # lognormal, normalised by its own min and max: starts at exactly 0
        assert wl.columns[j].min() == 0.0 and np.median(wl.columns[j]) < 0.1
    for j in (0, 2):
        assert abs(float(wl.columns[j].mean()) - 0.5) < 0.01
    for q in wl.queries:
        assert sorted(p[0] for p in q) == [0, 1, 2, 3]


def test_poisson_arrivals_rate_and_determinism():
    a = W.poisson_arrivals(1000.0, 20_000, seed=5)
    assert np.all(np.diff(a) > 0)
    gaps = np.diff(np.concatenate([[0.0], a]))
    assert abs(gaps.mean() * 1000.0 - 1.0) < 0.03  # mean gap 1 / rate (sd of the mean 0.7%)
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05  # exponential: sd equals the mean
    assert np.array_equal(a, W.poisson_arrivals(1000.0, 20_000, seed=5))
