"""CPU oracle for the multidimensional range query (MDRQ) — test infrastructure.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of
``bench.py`` may import this package. The GPU library does not import it and shares
no code with it; it exists to check that library.

The arithmetic lives in ``mdrq_oracle.c`` (plain C, compiled with gcc on first use
or by ``build()``); this module only marshals numpy arrays into it.

Semantics (Sec. 2.1): object i qualifies iff lb_j <= x_j[i] <= ub_j for every
constrained dimension j; unconstrained dimensions behave as [-inf, +inf]; the answer
is the ascending list of qualifying array indices (Sec. 2.2.4).

Two evaluations of that rule are exported, each pinned on its own: ``mdrq`` tests one
object at a time (the sequential scan of Sec. 2.2.4); ``mdrq_columnwise`` evaluates one
dimension at a time over its whole column and ANDs the per-object flags (the
vertically partitioned scan of Sec. 3.2). The second streams each column once, so it
answers full-size batches in a fraction of the first's time; the CPU baseline times
the first.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mdrq_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

F32 = 0
I32 = 1

_lock = threading.Lock()
_default = None


def compile_library(src: str, out: str) -> str:
    """Compile one oracle source file into a shared library at ``out``."""
    tmp = out + ".%d.tmp" % os.getpid()
    subprocess.check_call(
        ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-Wall", "-Wextra",
         "-o", tmp, src])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile ``mdrq_oracle.c`` into ``liboracle.so`` (in-tree) and return its path."""
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        compile_library(_SRC, _LIB)
    return _LIB


class Oracle:
    """ctypes view of one compiled oracle library."""

    def __init__(self, lib_path: str):
        lib = ctypes.CDLL(lib_path)
        for fn in (lib.oracle_mdrq, lib.oracle_mdrq_columnwise):
            fn.restype = ctypes.c_int64
            fn.argtypes = [
                ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int32),
                ctypes.c_uint32, ctypes.c_uint64,
                ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_double),
                ctypes.POINTER(ctypes.c_double), ctypes.c_uint32, ctypes.c_int,
                ctypes.POINTER(ctypes.POINTER(ctypes.c_uint32))]
        lib.oracle_free.restype = None
        lib.oracle_free.argtypes = [ctypes.POINTER(ctypes.c_uint32)]
        self._lib = lib

    def mdrq(self, columns, query, nthreads: int = 1) -> np.ndarray:
        return _mdrq(self._lib, self._lib.oracle_mdrq, columns, query, nthreads)

    def mdrq_columnwise(self, columns, query, nthreads: int = 1) -> np.ndarray:
        return _mdrq(self._lib, self._lib.oracle_mdrq_columnwise, columns, query, nthreads)


def default() -> Oracle:
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
    return _default


def _column_type(col: np.ndarray) -> int:
    if col.dtype == np.float32:
        return F32
    if col.dtype == np.int32:
        return I32
    raise TypeError("oracle columns must be float32 or int32, got %s" % col.dtype)


def _bound(col_dtype, v) -> float:
    """A bound as the column's own type sees it, carried exactly in a double."""
    if col_dtype == np.float32:
        return float(np.float32(v))
    return float(int(v))


def mdrq(columns, query, nthreads: int = 1) -> np.ndarray:
    """Answer one MDRQ with the row-at-a-time scan of the default oracle build.

    ``columns``: sequence of d 1-D arrays (float32 or int32), all of length n.
    ``query``: sequence of (dim, lo, hi) predicates; a dimension may repeat (its
    predicates are ANDed) and an empty sequence is the full-domain query.
    ``nthreads``: 1 for the sequential scan on one thread; p > 1 for p contiguous
    horizontal partitions scanned concurrently and concatenated in order (Sec. 3.1).
    Returns the ascending uint32 ids of the qualifying objects.
    """
    return default().mdrq(columns, query, nthreads)


def mdrq_columnwise(columns, query, nthreads: int = 1) -> np.ndarray:
    """The same answer as ``mdrq``, evaluated one dimension at a time (Sec. 3.2): per
    constrained dimension a flag per object over its column, the flags ANDed."""
    return default().mdrq_columnwise(columns, query, nthreads)


def _mdrq(lib, fn, columns, query, nthreads: int) -> np.ndarray:
    """Marshal one query into ``fn`` (an entry point of ``lib``)."""
    cols = [np.ascontiguousarray(c) for c in columns]
    d = len(cols)
    n = int(cols[0].shape[0]) if d else 0
    for c in cols:
        if c.ndim != 1 or c.shape[0] != n:
            raise ValueError("all columns must be 1-D of the same length")
    types = np.array([_column_type(c) for c in cols], dtype=np.int32)
    k = len(query)
    dims = np.array([int(p[0]) for p in query], dtype=np.uint32)
    for j in dims:
        if j >= d:
            raise ValueError("predicate on dimension %d of a %d-dimensional table" % (j, d))
    lo = np.array([_bound(cols[int(p[0])].dtype, p[1]) for p in query], dtype=np.float64)
    hi = np.array([_bound(cols[int(p[0])].dtype, p[2]) for p in query], dtype=np.float64)

    ptrs = (ctypes.c_void_p * max(d, 1))(*[c.ctypes.data for c in cols])
    out = ctypes.POINTER(ctypes.c_uint32)()
    cnt = fn(
        ptrs, types.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), d, n,
        dims.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
        lo.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        hi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), k, int(nthreads),
        ctypes.byref(out))
    if cnt < 0:
        raise RuntimeError("oracle_mdrq failed with status %d" % cnt)
    try:
        if cnt == 0:
            return np.zeros(0, dtype=np.uint32)
        return np.ctypeslib.as_array(out, shape=(cnt,)).copy()
    finally:
        lib.oracle_free(out)
