"""Checks that pin the MDRQ oracle to facts other than itself.

Each ``pin_*`` function takes ``f(columns, query, nthreads) -> ascending uint32 ids``
and raises AssertionError when ``f`` disagrees with what the paper or plain
mathematics fixes. They run against the real oracle (test_oracle_pins.py) and
against copies of it with a planted mistake (test_oracle_mutants.py), each of which
must fail at least one pin.
"""
from __future__ import annotations

import itertools
import json
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

INF = float("inf")


def _ids(a) -> list:
    return [int(v) for v in a]


# --------------------------------------------------------------------- brute force

def _inverted(col) -> dict:
    """value -> sorted list of rows holding exactly that value (bitwise for floats)."""
    inv = {}
    for i, v in enumerate(col.tolist()):
        inv.setdefault(v, []).append(i)
    return inv


def _brute(columns, domain_by_dim, query) -> list:
    """Answer a query without comparing any data value to a bound.

    Sec. 3.2 reading: per dimension, the set of matching rows is the union of the
    rows holding each domain value that lies in [lo, hi] (the domain is enumerated,
    not the data); the answer is the intersection over constrained dimensions.
    """
    n = columns[0].shape[0]
    rows = set(range(n))
    for (j, lo, hi) in query:
        hit = set()
        inv = _inverted(columns[j])
        for v in domain_by_dim[j]:
            if lo <= v <= hi:
                hit.update(inv.get(v, ()))
        rows &= hit
    return sorted(rows)


def pin_exhaustive_int(f) -> None:
    """Every interval combination over an int32 domain {0..3}, d=3, n=64 (plus the
    empty interval), complete- and partial-match, against the brute force above."""
    rng = np.random.default_rng(11)
    n, d = 64, 3
    cols = [rng.integers(0, 4, size=n, dtype=np.int32) for _ in range(d)]
    domain = [list(range(0, 4))] * d
    intervals = [(a, b) for a in range(4) for b in range(a, 4)] + [(2, 1)]
    count = 0
    for combo in itertools.product(intervals, repeat=d):
        q = [(j, lo, hi) for j, (lo, hi) in enumerate(combo)]
        assert _ids(f(cols, q, 1)) == _brute(cols, domain, q), q
        count += 1
    # partial-match: every single dimension and every pair
    for r in (1, 2):
        for dims in itertools.combinations(range(d), r):
            for combo in itertools.product(intervals, repeat=r):
                q = [(j, lo, hi) for j, (lo, hi) in zip(dims, combo)]
                assert _ids(f(cols, q, 1)) == _brute(cols, domain, q), q
    assert count == len(intervals) ** d


def pin_exhaustive_float_grid() -> tuple:
    """float32 values on a 1/8 grid in [-1/2, 1] with ties, -0.0 and +0.0 both present."""
    rng = np.random.default_rng(12)
    grid = np.arange(-4, 9, dtype=np.float32) / np.float32(8.0)
    n, d = 48, 2
    cols = [grid[rng.integers(0, grid.size, size=n)] for _ in range(d)]
    cols[0][3] = np.float32(-0.0)
    cols[1][5] = np.float32(-0.0)
    cols[0][7] = np.float32(0.0)
    return cols, grid


def pin_exhaustive_float(f) -> None:
    """All intervals with endpoints on the grid, +-inf and +-0.0, d=2, n=48."""
    cols, grid = pin_exhaustive_float_grid()
    ends = [float(v) for v in grid] + [-INF, INF, -0.0]
    domain = [sorted(set(float(v) for v in c.tolist())) for c in cols]
    intervals = [(a, b) for a in ends for b in ends if a <= b][::7] + [(0.5, 0.25)]
    for (a, b) in intervals:
        for (c, e) in intervals[::3]:
            q = [(0, a, b), (1, c, e)]
            assert _ids(f(cols, q, 1)) == _brute(cols, domain, q), q
    # [0, 0] holds both zeros: -0.0 == +0.0 (IEEE ordered compare)
    got = _ids(f(cols, [(0, 0.0, 0.0)], 1))
    assert 3 in got and 7 in got


def pin_numpy_single_dim(f) -> None:
    """One dimension: the answer is numpy.flatnonzero((x >= lo) & (x <= hi))."""
    rng = np.random.default_rng(13)
    x = rng.standard_normal(5000).astype(np.float32)
    xi = rng.integers(-50, 50, size=5000, dtype=np.int32)
    for lo, hi in [(-0.5, 0.25), (0.0, 0.0), (-INF, 0.1), (1.0, INF), (0.3, -0.3), (-INF, INF)]:
        lo32, hi32 = np.float32(lo), np.float32(hi)
        want = np.flatnonzero((x >= lo32) & (x <= hi32))
        assert _ids(f([x], [(0, lo, hi)], 1)) == _ids(want), (lo, hi)
    for lo, hi in [(-10, 10), (0, 0), (7, -7), (-2**31, 2**31 - 1)]:
        want = np.flatnonzero((xi >= lo) & (xi <= hi))
        assert _ids(f([xi], [(0, lo, hi)], 1)) == _ids(want), (lo, hi)


# --------------------------------------------------------------------- invariants

def _table(seed: int, n: int = 3000):
    rng = np.random.default_rng(seed)
    cols = [rng.random(n, dtype=np.float32) for _ in range(3)]
    cols.append(rng.integers(0, 20, size=n, dtype=np.int32))
    cols.append(np.floor(rng.random(n, dtype=np.float32) * 8).astype(np.float32) / 8)
    return cols


def _rand_query(rng, cols, k=None):
    d = len(cols)
    k = k or int(rng.integers(1, d + 1))
    q = []
    for j in sorted(rng.choice(d, size=k, replace=False).tolist()):
        c = cols[j]
        a, b = c[rng.integers(0, c.size)], c[rng.integers(0, c.size)]
        lo, hi = (a, b) if a <= b else (b, a)
        if c.dtype == np.int32:
            q.append((j, int(lo), int(hi)))
        else:
            q.append((j, float(lo), float(hi)))
    return q


def pin_invariants(f) -> None:
    cols = _table(21)
    n = cols[0].size
    d = len(cols)
    rng = np.random.default_rng(22)
    full = [(j, -INF, INF) if cols[j].dtype == np.float32 else (j, -2**31, 2**31 - 1)
            for j in range(d)]
    # full domain returns every id; the query with no predicates too (Sec. 2.1)
    assert _ids(f(cols, full, 1)) == list(range(n))
    assert _ids(f(cols, [], 1)) == list(range(n))
    for _ in range(25):
        q = _rand_query(rng, cols)
        r = _ids(f(cols, q, 1))
        s = set(r)
        assert r == sorted(s)  # ascending, no duplicates
        # partial-match == complete-match with [-inf, +inf] elsewhere (Sec. 2.1)
        qd = {p[0] for p in q}
        assert _ids(f(cols, q + [p for p in full if p[0] not in qd], 1)) == r
        # the answer is the intersection of the single-dimension answers (Sec. 3.2)
        inter = set(range(n))
        for p in q:
            inter &= set(_ids(f(cols, [p], 1)))
        assert s == inter
        # the order of the dimensions does not matter (Sec. 2.2.4)
        assert _ids(f(cols, q[::-1], 1)) == r
        # an empty interval on any one dimension gives no answer
        j, lo, hi = q[int(rng.integers(0, len(q)))]
        if lo < hi:
            assert _ids(f(cols, q + [(j, hi, lo)], 1)) == []
        # widening is monotone: a superset
        wide = [(jj, lo2 - (0.1 if cols[jj].dtype == np.float32 else 1),
                 hi2 + (0.1 if cols[jj].dtype == np.float32 else 1)) for (jj, lo2, hi2) in q]
        assert s <= set(_ids(f(cols, wide, 1)))
        # splitting an interval at v gives a disjoint union of the two answers
        j, lo, hi = q[0]
        c = cols[j]
        if c.dtype == np.int32:
            v = (lo + hi) // 2
            left, right = (j, lo, v), (j, v + 1, hi)
        else:
            v = np.float32((lo + hi) / 2)
            left = (j, lo, float(v))
            right = (j, float(np.nextafter(v, np.float32(INF))), hi)
        a = set(_ids(f(cols, [left] + q[1:], 1)))
        b = set(_ids(f(cols, [right] + q[1:], 1)))
        assert not (a & b) and (a | b) == s
        # horizontal partitions concatenated in order equal the whole (Sec. 3.1)
        cut = int(rng.integers(0, n + 1))
        lo_part = _ids(f([c_[:cut] for c_ in cols], q, 1))
        hi_part = [i + cut for i in _ids(f([c_[cut:] for c_ in cols], q, 1))]
        assert lo_part + hi_part == r
        # the threaded scan (p contiguous partitions) gives the same list
        assert _ids(f(cols, q, 3)) == r
        # a repeated dimension ANDs its predicates
        j, lo, hi = q[-1]
        assert set(_ids(f(cols, q + [(j, lo, hi)], 1))) == s
    # a point query returns exactly the rows equal to that point (duplicates included)
    for r0 in rng.integers(0, n, size=10).tolist():
        q = [(j, cols[j][r0].item(), cols[j][r0].item()) for j in (3, 4)]
        want = [i for i in range(n) if cols[3][i] == cols[3][r0] and cols[4][i] == cols[4][r0]]
        got = _ids(f(cols, q, 1))
        assert got == want and r0 in got and len(got) > 1


def pin_degenerate(f) -> None:
    """n = 0 answers nothing; n = 1 answers [0] or nothing."""
    e = np.zeros(0, dtype=np.float32)
    assert _ids(f([e], [(0, 0.0, 1.0)], 1)) == []
    assert _ids(f([e], [], 4)) == []
    one = np.array([0.5], dtype=np.float32)
    assert _ids(f([one], [(0, 0.5, 0.5)], 1)) == [0]
    assert _ids(f([one], [(0, 0.6, 1.0)], 2)) == []


# --------------------------------------------------------------------- the paper's numbers

def random_pair_closed_form(m: int, n: int) -> tuple:
    """Mean and standard deviation of the selectivity of a random-pair query on n
    uniform objects in m independent dimensions (Sec. 7.2.1 queries).

    The two objects that define the bounds always qualify (closed intervals); each
    other object qualifies with probability prod_j |a_j - b_j|, whose mean over the
    pair is (1/3)^m and whose second moment is (1/6)^m (E|a-b| = 1/3,
    E(a-b)^2 = 1/6 for independent uniforms)."""
    mean_p = (1.0 / 3.0) ** m
    var_p = (1.0 / 6.0) ** m - (1.0 / 9.0) ** m
    mean = (2.0 + (n - 2) * mean_p) / n
    sd = (n - 2) / n * math.sqrt(var_p)
    return mean, sd


def pin_random_pair_expectation(f) -> None:
    """Per query, E[count | bounds] = 2 + (n - 2) * prod_j (hi_j - lo_j) on uniform
    data; the total over many queries must agree within binomial noise."""
    rng = np.random.default_rng(31)
    n, m = 20000, 5
    cols = [rng.random(n, dtype=np.float32) for _ in range(m)]
    total, expect, var = 0, 0.0, 0.0
    for _ in range(300):
        a, b = rng.integers(0, n, size=2)
        q = []
        p = 1.0
        for j in range(m):
            lo, hi = sorted((float(cols[j][a]), float(cols[j][b])))
            q.append((j, lo, hi))
            p *= hi - lo
        got = _ids(f(cols, q, 1))
        assert a in got and b in got  # both defining objects lie inside the closed box
        total += len(got)
        expect += (2 if a != b else 1) + (n - 2) * p
        var += (n - 2) * p * (1 - p)
    assert abs(total - expect) < 5 * math.sqrt(var) + 5, (total, expect, var)


def pin_paper_high_dim_selectivity(f) -> None:
    """Sec. 7.4.1: with more than 10 dimensions the random-pair selectivity on 1M
    uniform objects is 0.0002% — exactly the two defining objects."""
    gold = json.load(open(os.path.join(GOLDEN, "random_pair_selectivity.json")))
    n = gold["n"]
    rng = np.random.default_rng(32)
    m = 20
    cols = [rng.random(n, dtype=np.float32) for _ in range(m)]
    sels = []
    for _ in range(6):
        a, b = rng.integers(0, n, size=2)
        q = [(j, *sorted((float(cols[j][a]), float(cols[j][b])))) for j in range(m)]
        sels.append(100.0 * len(f(cols, q, 4)) / n)
    # each answer holds exactly the two defining objects: 2 / 1M = 0.0002%
    assert all(abs(s - gold["m_gt10"]["mean_pct"]) < 1e-12 for s in sels), sels


def pin_paper_5d_selectivity(f) -> None:
    """Sec. 7.4.1: random-pair queries on uniform 5-D data have mean selectivity 0.4%
    and standard deviation 1.1% (both rounded as printed)."""
    gold = json.load(open(os.path.join(GOLDEN, "random_pair_selectivity.json")))
    rng = np.random.default_rng(33)
    n, m, nq = 100_000, 5, 1500
    cols = [rng.random(n, dtype=np.float32) for _ in range(m)]
    sels = []
    for _ in range(nq):
        a, b = rng.integers(0, n, size=2)
        q = [(j, *sorted((float(cols[j][a]), float(cols[j][b])))) for j in range(m)]
        sels.append(100.0 * len(f(cols, q, 4)) / n)
    mean, sd = float(np.mean(sels)), float(np.std(sels))
    se = gold["m5"]["sd_pct"] / math.sqrt(nq)
    assert abs(mean - gold["m5"]["mean_pct"]) < 0.05 + 4 * se, mean
    assert 0.8 < sd / gold["m5"]["sd_pct"] < 1.25, sd


ALL_PINS = [pin_exhaustive_int, pin_exhaustive_float, pin_numpy_single_dim, pin_invariants,
            pin_degenerate, pin_random_pair_expectation, pin_paper_high_dim_selectivity,
            pin_paper_5d_selectivity]
