"""The C-ABI library loads, exports every symbol its header declares, and rejects bad
arguments before touching the GPU (no compute calls here; runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_1801_03644_gb300 import build as B
from paper_1801_03644_gb300 import mdrq

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return mdrq.lib()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(mdrq_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert {"mdrq_load_columns", "mdrq_query", "mdrq_query_batch", "mdrq_free"} <= set(names)
    for name in names:
        assert hasattr(L, name), name
    assert set(mdrq.EXPORTS) <= set(names)


def test_status_strings(L):
    assert L.mdrq_status_string(0) == b"ok"
    assert b"NaN" in L.mdrq_status_string(-6)
    assert L.mdrq_status_string(-99) == b"unknown status"


def test_null_safe_calls(L):
    L.mdrq_free(None)
    assert L.mdrq_table_rows(None) == 0
    assert L.mdrq_table_dims(None) == 0
    a, b = ctypes.c_uint64(7), ctypes.c_uint64(7)
    L.mdrq_last_scan_stats(None, ctypes.byref(a), ctypes.byref(b))
    assert a.value == 0 and b.value == 0


def test_load_rejects_bad_arguments_before_cuda(L):
    h = ctypes.c_void_p()
    types = (ctypes.c_int32 * 2)(0, 1)
    cols = (ctypes.c_void_p * 2)(16, 32)
    # d = 0
    assert L.mdrq_load_columns(cols, types, 0, 10, 1, None, ctypes.byref(h)) == mdrq.E_INVAL
    # n >= 2^32 (ids are uint32)
    assert L.mdrq_load_columns(cols, types, 2, 1 << 32, 1, None, ctypes.byref(h)) == mdrq.E_INVAL
    # unknown column type
    bad = (ctypes.c_int32 * 2)(0, 7)
    assert L.mdrq_load_columns(cols, bad, 2, 10, 1, None, ctypes.byref(h)) == mdrq.E_INVAL
    # device columns must be 16-byte aligned
    mis = (ctypes.c_void_p * 2)(16, 36)
    assert L.mdrq_load_columns(mis, types, 2, 10, 1, None, ctypes.byref(h)) == mdrq.E_INVAL
    # null column with rows
    nul = (ctypes.c_void_p * 2)(16, None)
    assert L.mdrq_load_columns(nul, types, 2, 10, 1, None, ctypes.byref(h)) == mdrq.E_INVAL
    # no output handle
    assert L.mdrq_load_columns(cols, types, 2, 10, 1, None, None) == mdrq.E_INVAL
    assert h.value is None


def test_query_rejects_null_table(L):
    cnt = ctypes.c_uint64(0)
    p = (mdrq.Pred * 1)()
    assert L.mdrq_query(None, p, 1, None, 0, ctypes.byref(cnt), 1, None) == mdrq.E_INVAL
    off = (ctypes.c_uint64 * 2)()
    assert L.mdrq_query_batch(None, None, 0, None, 0, off, 1, None) == mdrq.E_INVAL


def test_bound_encoding():
    p = mdrq.encode_query([(1, -0.0, 0.5), (0, -5, 7)], [mdrq.I32, mdrq.F32])
    assert p[0].dim == 1 and p[0].lo == 0x80000000 and p[0].hi == 0x3F000000
    assert p[1].dim == 0 and p[1].lo == 0xFFFFFFFB and p[1].hi == 7
    with pytest.raises(ValueError):
        mdrq.encode_query([(2, 0, 1)], [mdrq.F32, mdrq.F32])
    with pytest.raises(ValueError):
        mdrq.encode_query([(0, 0, 2**31)], [mdrq.I32])
