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


def test_static_entry_checks_arguments_before_cuda(L):
    """mdrq_query_static rejects every bad argument, and answers a provably empty query
    (an empty interval, or an empty table) with count 0, before its first CUDA call.
    The column addresses are fake, aligned and never dereferenced."""
    def call(cols, types, d, n, preds, count=True):
        c = (ctypes.c_void_p * max(1, len(cols)))(*cols)
        t = (ctypes.c_int32 * max(1, len(types)))(*types)
        p = mdrq.encode_query(preds, types) if preds else (mdrq.Pred * 1)()
        cnt = ctypes.c_uint64(12345)
        st = L.mdrq_query_static(c, t, d, n, p, len(preds), None, 0,
                                 ctypes.byref(cnt) if count else None, None)
        return st, cnt.value

    cols, types = [0x10000, 0x20000], [mdrq.F32, mdrq.I32]
    nan = float("nan")
    assert call(cols, types, 2, mdrq.STATIC_MAX_ROWS + 1, [(0, 0.0, 1.0)])[0] == mdrq.E_INVAL
    assert call([0x10004, 0x20000], types, 2, 10, [(0, 0.0, 1.0)])[0] == mdrq.E_INVAL  # misaligned
    assert call([0, 0x20000], types, 2, 10, [(0, 0.0, 1.0)])[0] == mdrq.E_INVAL        # null column
    assert call(cols, [mdrq.F32, 7], 2, 10, [(0, 0.0, 1.0)])[0] == mdrq.E_INVAL        # unknown type
    assert call(cols, types, 0, 10, [])[0] == mdrq.E_INVAL                             # d = 0
    assert call(cols, types, 2, 10, [(0, nan, 1.0)])[0] == mdrq.E_INVAL                # NaN bound
    assert call(cols, types, 2, 10, [(0, 0.0, 1.0)], count=False)[0] == mdrq.E_INVAL   # count NULL
    bad_dim = mdrq.encode_query([(0, 0.0, 1.0)], types)
    bad_dim[0].dim = 2
    cnt = ctypes.c_uint64(0)
    assert L.mdrq_query_static((ctypes.c_void_p * 2)(*cols), (ctypes.c_int32 * 2)(*types), 2, 10, bad_dim, 1,
                               None, 0, ctypes.byref(cnt), None) == mdrq.E_INVAL
    bad_dim[0].dim = 0
    bad_dim[0].reserved = 1
    assert L.mdrq_query_static((ctypes.c_void_p * 2)(*cols), (ctypes.c_int32 * 2)(*types), 2, 10, bad_dim, 1,
                               None, 0, ctypes.byref(cnt), None) == mdrq.E_INVAL
    # more than 128 distinct constrained dimensions
    many = [0x10000 * (j + 1) for j in range(130)]
    ftypes = [mdrq.F32] * 130
    assert call(many, ftypes, 130, 10, [(j, 0.0, 1.0) for j in range(129)])[0] == mdrq.E_INVAL
    # provably empty: answered on the host with count 0
    assert call(cols, types, 2, 10, [(0, 1.0, 0.0)]) == (mdrq.OK, 0)
    assert call(cols, types, 2, 10, [(1, 5, 9), (1, 10, 20)]) == (mdrq.OK, 0)  # repeated dim, disjoint
    assert call(cols, types, 2, 0, [(0, 0.0, 1.0)]) == (mdrq.OK, 0)            # empty table


def test_every_handle_call_rejects_null(L):
    """Each call taking a table, server or prepared-batch handle returns MDRQ_E_INVAL for
    a NULL handle (stop and free are no-ops), before any CUDA call."""
    u64, u32, dbl, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_int
    a, b, c = u64(0), u64(0), u64(0)
    s, d1, d2 = u32(0), dbl(0), dbl(0)
    p = (mdrq.Pred * 1)()
    q = (mdrq.QDesc * 1)()
    h = ctypes.c_void_p()
    tick = (u64 * 1)(1)
    st = (i32 * 1)()
    tune = mdrq.Tuning()
    ms = dbl(0)
    E = mdrq.E_INVAL
    assert L.mdrq_set_batch_mode(None, mdrq.BATCH_PLAIN) == E
    assert L.mdrq_learn(None, (u32 * 1)(0), 1, mdrq.MODEL_PLA, None) == E
    assert L.mdrq_learn_info(None, ctypes.byref(a), ctypes.byref(s), ctypes.byref(d1)) == E
    assert L.mdrq_learn_window_rows(None, ctypes.byref(a), ctypes.byref(b)) == E
    assert L.mdrq_server_start(None, 1 << 20, 16, ctypes.byref(h)) == E and h.value is None
    assert L.mdrq_server_submit(None, p, 1, ctypes.byref(a)) == E
    assert L.mdrq_server_submit_batch(None, q, 1, tick) == E
    assert L.mdrq_server_wait(None, 1, 0, None, ctypes.byref(a), ctypes.byref(d1)) == E
    assert L.mdrq_server_wait_many(None, tick, 1, 0, st, None, None, 0) == E
    assert L.mdrq_server_release(None, 1) == E
    assert L.mdrq_server_stats(None, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d1),
                               ctypes.byref(d2)) == E
    assert L.mdrq_server_stop(None) == mdrq.OK
    off = (u64 * 2)()
    assert L.mdrq_prepare_batch(None, q, 1, None, 0, off, None, ctypes.byref(h)) == E and h.value is None
    assert L.mdrq_prepared_launch(None, None) == E
    assert L.mdrq_prepared_wait(None, off, None) == E
    assert L.mdrq_prepared_kernels(None, ctypes.byref(a)) == E
    L.mdrq_prepared_free(None)
    assert L.mdrq_set_shared_config(None, 0, 0) == E
    assert L.mdrq_set_shared_bits_budget(None, 0) == E
    assert L.mdrq_autotune(None, q, 1, None, ctypes.byref(tune)) == E
    assert L.mdrq_set_zone_maps(None, mdrq.ZONES_AUTO) == E
    assert L.mdrq_zone_map_info(None, 0, None, None) == E
    assert L.mdrq_zone_scan_info(None, ctypes.byref(a), ctypes.byref(b)) == E
    assert L.mdrq_scan_timing(None, 1) == E
    assert L.mdrq_scan_timing_read(None, ctypes.byref(ms), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), 0) == E
    assert L.mdrq_inject_fault(None, mdrq.FAULT_NOMEM, 0) == E
    assert L.mdrq_inject_fault(None, mdrq.FAULT_STAGE_NOMEM, 0) == E
    k, empty = u32(0), i32(0)
    assert L.mdrq_explain_query(None, p, 1, p, 1, ctypes.byref(k), ctypes.byref(empty)) == E
    assert L.mdrq_learn_search_info(None, ctypes.byref(a), ctypes.byref(b)) == E
    desc = mdrq.ModelDesc()
    assert L.mdrq_learn_export(None, ctypes.byref(desc), None, None, None, None, 0) == E
    assert L.mdrq_set_host_answers(None, mdrq.HOST_AUTO) == E
    assert L.mdrq_set_shared_codes(None, 1) == E
    assert L.mdrq_set_output_order(None, mdrq.ORDER_AUTO) == E
    assert L.mdrq_set_key_cells(None, 0, None, 0) == E
