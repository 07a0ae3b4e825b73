"""Seeded synthetic tables and range queries shaped like the paper's workloads.

This module is the one thing the GPU library and the CPU oracle share: it makes
their *inputs*. It holds none of the query method's arithmetic (no predicate is
evaluated here), so both sides stay independent.

The paper's own datasets (GMRQB, SYNT-CLUST's generator, POWER; Sec. 6, 7.2) are
not available; these generators stand in for them at GPU scale.

RNG: numpy PCG64, ``default_rng(SeedSequence([config_id, stream]))``; stream 0 draws
the table column by column in dimension order, stream 1 the queries, stream 2 the
row sample used to place query bounds at quantiles. The small uniform table is the
exception: it is ``default_rng(0).random((3, n), dtype=float32)``.

A query is a list of ``(dim, lo, hi)`` predicates; ``lo``/``hi`` are Python numbers
that are exact values of the column's type (float32 or int32). Dimensions absent
from the list are unconstrained (partial-match, Sec. 2.1).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

ONE_BELOW = float(np.nextafter(np.float32(1.0), np.float32(0.0)))  # 0.99999994


def rng_for(config_id: int, stream: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([config_id, stream]))


@dataclasses.dataclass
class Workload:
    name: str
    columns: list          # d 1-D numpy arrays (float32 / int32), length n
    queries: list          # list of queries; a query is a list of (dim, lo, hi)
    recipe: str            # one line: how the inputs were drawn
    key_bounds: list = None  # Z-sorted tables: per key column the 255 cell bounds, or None

    @property
    def n(self) -> int:
        return int(self.columns[0].shape[0]) if self.columns else 0

    @property
    def d(self) -> int:
        return len(self.columns)


# ----------------------------------------------------------------------------- columns

def uniform_column(rng: np.random.Generator, n: int) -> np.ndarray:
    """float32 uniform on [0, 1)."""
    return rng.random(n, dtype=np.float32)


def cluster_mixture_columns(rng: np.random.Generator, n: int, d: int, n_clusters: int = 20,
                            sigma: float = 0.02, chunk: int = 1 << 24) -> list:
    """d float32 columns drawn jointly from a mixture of Gaussian clusters.

    Each row picks one cluster c uniformly; every column j takes
    centre[c, j] + sigma * N(0, 1), clipped to [0, nextafter(1, 0)]. Centres are
    uniform on [0, 1).
    """
    centres = rng.random((n_clusters, d), dtype=np.float32)
    cid = rng.integers(0, n_clusters, size=n, dtype=np.uint8)
    cols = []
    s = np.float32(sigma)
    for j in range(d):
        col = np.empty(n, dtype=np.float32)
        for a in range(0, n, chunk):
            b = min(n, a + chunk)
            z = rng.standard_normal(b - a, dtype=np.float32)
            np.multiply(z, s, out=z)
            np.add(z, centres[cid[a:b], j], out=z)
            np.clip(z, np.float32(0.0), np.float32(ONE_BELOW), out=z)
            col[a:b] = z
        cols.append(col)
    return cols


def zipf_column(rng: np.random.Generator, n: int, s: float = 1.2, vmax: int = 1_000_000,
                chunk: int = 1 << 22) -> np.ndarray:
    """int32 bounded Zipf: P(v) proportional to v^-s for v in 1..vmax (inverse CDF)."""
    w = np.arange(1, vmax + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    out = np.empty(n, dtype=np.int32)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        u = rng.random(b - a)
        v = np.searchsorted(cdf, u, side="right") + 1
        np.minimum(v, vmax, out=v)
        out[a:b] = v
    return out


def categorical_column(rng: np.random.Generator, n: int, ncat: int = 64) -> np.ndarray:
    """int32 uniform over {0 .. ncat-1}."""
    return rng.integers(0, ncat, size=n, dtype=np.int32)


# ----------------------------------------------------------------------------- queries

def quantile_samples(columns: list, rng: np.random.Generator, sample: int = 1 << 20) -> list:
    """Sorted per-column samples (the whole column when n <= sample) for placing bounds."""
    n = int(columns[0].shape[0])
    if n <= sample:
        return [np.sort(c) for c in columns]
    idx = rng.integers(0, n, size=sample)
    return [np.sort(c[idx]) for c in columns]


def _quantile(sorted_sample: np.ndarray, p: float):
    m = sorted_sample.shape[0]
    i = min(m - 1, max(0, int(math.floor(p * (m - 1)))))
    return sorted_sample[i]


def _as_bound(col_dtype, v):
    if col_dtype == np.float32:
        return float(np.float32(v))
    return int(v)


def target_selectivity_query(samples: list, dtypes: list, dims, s: float,
                             rng: np.random.Generator) -> list:
    """Predicates on ``dims`` aiming at overall selectivity ``s``.

    Each dimension gets the share s_j = s^(1/k) and the interval between the
    sample quantiles u and u + s_j, with u uniform on [0, 1 - s_j]. On correlated
    dimensions the achieved selectivity differs from ``s`` (Sec. 2.1); it is
    measured, never assumed.
    """
    k = len(dims)
    sj = s ** (1.0 / k)
    q = []
    for j in dims:
        u = rng.uniform(0.0, max(0.0, 1.0 - sj))
        lo = _quantile(samples[j], u)
        hi = _quantile(samples[j], min(1.0, u + sj))
        q.append((int(j), _as_bound(dtypes[j], lo), _as_bound(dtypes[j], hi)))
    return q


def log_uniform(rng: np.random.Generator, lo: float, hi: float) -> float:
    return float(math.exp(rng.uniform(math.log(lo), math.log(hi))))


def random_pair_queries(columns: list, nq: int, rng: np.random.Generator) -> list:
    """Complete-match queries from two random objects (Sec. 7.2.1).

    Per dimension the interval runs from the smaller to the larger of the two
    objects' values, so it is never empty.
    """
    n = int(columns[0].shape[0])
    qs = []
    for _ in range(nq):
        a, b = rng.integers(0, n, size=2)
        q = []
        for j, c in enumerate(columns):
            va, vb = c[a], c[b]
            lo, hi = (va, vb) if va <= vb else (vb, va)
            q.append((j, _as_bound(c.dtype, lo), _as_bound(c.dtype, hi)))
        qs.append(q)
    return qs


# ----------------------------------------------------------------------------- configurations

UNIFORM_SMALL_WIDTH = 0.01 ** (1.0 / 3.0)  # 0.21544346900318834: 1% over 3 dims


def uniform_small(n: int = 1_000_000, nq: int = 100) -> Workload:
    """1M x 3 float32 uniform on [0,1) from seed 0; complete-match queries of width
    0.01^(1/3) per dimension at a uniform offset (about 1% selectivity)."""
    cols = list(np.random.default_rng(0).random((3, n), dtype=np.float32))
    rng = rng_for(1, 1)
    w = UNIFORM_SMALL_WIDTH
    qs = []
    for _ in range(nq):
        q = []
        for j in range(3):
            lo = rng.uniform(0.0, 1.0 - w)
            q.append((j, float(np.float32(lo)), float(np.float32(lo + w))))
        qs.append(q)
    return Workload("uniform_1Mx3_f32", cols, qs,
                    "n=%d d=3 f32 U[0,1) seed 0; %d complete-match queries, width "
                    "0.01^(1/3) at U[0,1-w] offsets" % (n, nq))


def mixed_clustered(n: int = 100_000_000, nq: int = 1024, sel_range=(1e-5, 0.2)) -> Workload:
    """n x 8 float32: dims 0-3 uniform on [0,1), dims 4-7 a joint mixture of 20
    Gaussian clusters (sigma 0.02, centres uniform, clipped to [0,1)). Partial-match
    queries on 2..8 random dims, target selectivity log-uniform in ``sel_range``."""
    rng = rng_for(2, 0)
    cols = [uniform_column(rng, n) for _ in range(4)]
    cols += cluster_mixture_columns(rng, n, 4)
    dtypes = [c.dtype for c in cols]
    samples = quantile_samples(cols, rng_for(2, 2))
    qrng = rng_for(2, 1)
    qs = []
    for _ in range(nq):
        k = int(qrng.integers(2, 9))
        dims = sorted(qrng.choice(8, size=k, replace=False).tolist())
        s = log_uniform(qrng, *sel_range)
        qs.append(target_selectivity_query(samples, dtypes, dims, s, qrng))
    return Workload("mixed_clustered_%dx8_f32" % n, cols, qs,
                    "n=%d d=8 f32 (4 U[0,1), 4 joint 20-cluster mixture sigma 0.02); %d "
                    "partial-match queries, k~U{2..8}, target sel log-uniform [%g, %g]"
                    % (n, nq, sel_range[0], sel_range[1]))


def skewed_mixed_types(n: int = 50_000_000, nq: int = 256, sel_range=(1e-6, 0.5),
                       empty_fraction: float = 0.05) -> Workload:
    """n x 32: 16 float32 uniform on [0,1), 8 int32 Zipf(1.2) over 1..10^6, 8 int32
    categorical over 64 values. Queries on 3..12 random dims, target selectivity
    log-uniform in ``sel_range``; a fraction are made empty on purpose (one int
    interval outside the domain, or lo > hi)."""
    rng = rng_for(3, 0)
    cols = [uniform_column(rng, n) for _ in range(16)]
    cols += [zipf_column(rng, n) for _ in range(8)]
    cols += [categorical_column(rng, n) for _ in range(8)]
    dtypes = [c.dtype for c in cols]
    samples = quantile_samples(cols, rng_for(3, 2))
    qrng = rng_for(3, 1)
    qs = []
    for _ in range(nq):
        k = int(qrng.integers(3, 13))
        dims = sorted(qrng.choice(32, size=k, replace=False).tolist())
        s = log_uniform(qrng, *sel_range)
        q = target_selectivity_query(samples, dtypes, dims, s, qrng)
        if qrng.random() < empty_fraction:
            ints = [i for i, p in enumerate(q) if p[0] >= 16]
            if ints:
                i = ints[int(qrng.integers(0, len(ints)))]
                j = q[i][0]
                if qrng.random() < 0.5:
                    q[i] = (j, 2_000_000, 3_000_000)
                else:
                    q[i] = (j, q[i][2] + 1, q[i][1])  # lo > hi
            else:
                j, lo, hi = q[0]
                q[0] = (j, hi, lo) if lo != hi else (j, 2.0, 3.0)
        qs.append(q)
    return Workload("skewed_mixed_%dx32" % n, cols, qs,
                    "n=%d d=32 (16 f32 U[0,1), 8 i32 Zipf(1.2) 1..1e6, 8 i32 cat 64); %d "
                    "queries, k~U{3..12}, target sel log-uniform [%g, %g], %.0f%% forced empty"
                    % (n, nq, sel_range[0], sel_range[1], 100 * empty_fraction))


def zorder_cell(v: np.ndarray, bounds=None) -> np.ndarray:
    """8-bit cell of a value for the Z-order layout: with ``bounds`` (255 ascending
    float32 values) the number of bounds <= v, else clamp(floor(v * 256), 0, 255)."""
    v = np.asarray(v, dtype=np.float32)
    if bounds is not None:
        return np.searchsorted(np.asarray(bounds, dtype=np.float32), v, side="right").astype(np.uint32)
    c = np.floor(v * np.float32(256.0))
    return np.clip(c, 0, 255).astype(np.uint32)


def quantile_cell_bounds(column: np.ndarray, rng: np.random.Generator, sample: int = 1 << 20) -> np.ndarray:
    """255 cell bounds at the 1/256 .. 255/256 quantiles of a sample of the column, so
    that each of the 256 cells holds about as many rows (float32, ascending)."""
    n = column.shape[0]
    s = np.sort(column[rng.integers(0, n, size=min(sample, max(1, n)))] if n else column)
    if s.size == 0:
        return np.linspace(0, 1, 257, dtype=np.float32)[1:-1]
    idx = (np.arange(1, 256) * s.size) // 256
    return s[np.minimum(idx, s.size - 1)].astype(np.float32)


def zorder_key(columns: list, bounds=None) -> np.ndarray:
    """32-bit Morton key over up to 4 columns: bit 4b + j of the key is bit b of column
    j's 8-bit cell (dimension 0 least significant in each nibble); ``bounds``: per
    column the cell bounds of ``zorder_cell``, or None for equal-width cells."""
    key = np.zeros(columns[0].shape[0], dtype=np.uint32)
    for j, c in enumerate(columns):
        cell = zorder_cell(c, None if bounds is None else bounds[j])
        for b in range(8):
            key |= ((cell >> np.uint32(b)) & np.uint32(1)) << np.uint32(4 * b + j)
    return key


def zorder_learned(n: int = 200_000_000, nq: int = 4096, sel_range=(1e-4, 0.05),
                   chunk: int = 1 << 24) -> Workload:
    """n x 4 float32: dims 0 and 2 uniform on [0,1); dims 1 and 3 lognormal(0, 1)
    normalised to [0,1) by (y - min) / (max - min) and clipped to [0, 0.99999994]. Rows
    are sorted (stably) by the 32-bit Z-order key of the 4 dims over quantile cells
    (each dimension's 256 cells cut at the quantiles of a 2^20-row sample, so that every
    cell holds about n / 256 rows; ``key_bounds`` of the result). Complete-match
    queries, target selectivity log-uniform in ``sel_range``, s^(1/4) per dimension by
    quantile."""
    rng = rng_for(4, 0)
    cols = []
    for j in range(4):
        if j % 2 == 0:
            cols.append(uniform_column(rng, n))
        else:
            y = np.empty(n, dtype=np.float64)
            for a in range(0, n, chunk):
                b = min(n, a + chunk)
                y[a:b] = rng.lognormal(0.0, 1.0, size=b - a)
            lo, hi = y.min(), y.max()
            span = hi - lo if hi > lo else 1.0
            x = ((y - lo) / span).astype(np.float32)
            del y
            np.clip(x, np.float32(0.0), np.float32(ONE_BELOW), out=x)
            cols.append(x)
    crng = rng_for(4, 3)
    bounds = [quantile_cell_bounds(c, crng) for c in cols]
    key = zorder_key(cols, bounds)
    order = np.argsort(key, kind="stable")
    del key
    cols = [c[order] for c in cols]
    del order
    dtypes = [c.dtype for c in cols]
    samples = quantile_samples(cols, rng_for(4, 2))
    qrng = rng_for(4, 1)
    qs = []
    for _ in range(nq):
        s = log_uniform(qrng, *sel_range)
        qs.append(target_selectivity_query(samples, dtypes, [0, 1, 2, 3], s, qrng))
    return Workload("zorder_%dx4_f32" % n, cols, qs,
                    "n=%d d=4 f32 (2 U[0,1), 2 normalised lognormal(0,1)), rows sorted by the "
                    "32-bit Z-order key over quantile cells; %d complete-match queries, target sel "
                    "log-uniform [%g, %g]" % (n, nq, sel_range[0], sel_range[1]), key_bounds=bounds)


def serving_table(n: int = 20_000_000, nq: int = 20_000, sel_range=(1e-5, 0.1)) -> Workload:
    """n x 16 float32: dims 0-7 uniform on [0,1), dims 8-15 the joint 20-cluster
    mixture of ``mixed_clustered``. Queries constrain 1..16 random dims, target
    selectivity log-uniform in ``sel_range`` (the serving stream draws from them)."""
    rng = rng_for(5, 0)
    cols = [uniform_column(rng, n) for _ in range(8)]
    cols += cluster_mixture_columns(rng, n, 8)
    dtypes = [c.dtype for c in cols]
    samples = quantile_samples(cols, rng_for(5, 2))
    qrng = rng_for(5, 1)
    qs = []
    for _ in range(nq):
        k = int(qrng.integers(1, 17))
        dims = sorted(qrng.choice(16, size=k, replace=False).tolist())
        s = log_uniform(qrng, *sel_range)
        qs.append(target_selectivity_query(samples, dtypes, dims, s, qrng))
    return Workload("serving_%dx16_f32" % n, cols, qs,
                    "n=%d d=16 f32 (8 U[0,1), 8 joint 20-cluster mixture sigma 0.02); %d queries, "
                    "k~U{1..16}, target sel log-uniform [%g, %g]" % (n, nq, sel_range[0], sel_range[1]))


def poisson_arrivals(rate_per_s: float, count: int, seed: int = 0) -> np.ndarray:
    """Arrival times (seconds from 0) of an open-loop Poisson stream."""
    gaps = rng_for(50 + seed, 0).exponential(1.0 / rate_per_s, size=count)
    return np.cumsum(gaps)


def paper_uniform(n: int, d: int, nq: int, seed: int = 7) -> Workload:
    """SYNT-UNI (Sec. 7.2.1): n x d float32 uniform on [0,1), random-pair queries."""
    rng = rng_for(100 + seed, 0)
    cols = [uniform_column(rng, n) for _ in range(d)]
    qs = random_pair_queries(cols, nq, rng_for(100 + seed, 1))
    return Workload("synt_uni_%dx%d" % (n, d), cols, qs,
                    "n=%d d=%d f32 U[0,1); %d random-pair complete-match queries" % (n, d, nq))
