"""Python binding of the MDRQ scan library (``libmdrq.so``, C ABI in ``include/mdrq.h``).

Argument marshalling only: every step of a query runs in the library's CUDA kernels.
PyTorch provides device memory and streams. There is no CPU fallback: if the library
is missing or no GPU is present, the calls raise.

Ids are uint32 row indices (ascending per query). Device answers are returned in
``torch.int32`` tensors holding the uint32 bit patterns (identical for n < 2^31); use
``as_uint32_numpy`` to read them as uint32 on the host.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmdrq.so")

F32, I32 = 0, 1
OK, E_INVAL, E_NOMEM, E_CUDA, E_CAPACITY, E_TIMEOUT, E_NAN = 0, -1, -2, -3, -4, -5, -6


class MDRQError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__("%s failed: %s (status %d)" % (what, status_string(status), status))
        self.status = status


class Pred(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("lo", ctypes.c_uint32), ("hi", ctypes.c_uint32)]


class Tuning(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("unit_rows", ctypes.c_uint32), ("image_kib", ctypes.c_uint32),
                ("candidates", ctypes.c_uint32), ("plain_ms", ctypes.c_double),
                ("shared_default_ms", ctypes.c_double), ("shared_ms", ctypes.c_double)]


class ModelDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("segments", ctypes.c_uint32), ("mlp_params", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("key_min", ctypes.c_uint64), ("key_inv", ctypes.c_float),
                ("reserved2", ctypes.c_float), ("max_error", ctypes.c_uint64)]


class QDesc(ctypes.Structure):
    _fields_ = [("preds", ctypes.POINTER(Pred)), ("npreds", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


_lib = None

EXPORTS = ["mdrq_load_columns", "mdrq_query", "mdrq_query_batch", "mdrq_free",
           "mdrq_status_string", "mdrq_table_rows", "mdrq_table_dims", "mdrq_last_scan_stats",
           "mdrq_scan_timing", "mdrq_scan_timing_read", "mdrq_query_static",
           "mdrq_inject_fault", "mdrq_set_batch_mode", "mdrq_learn", "mdrq_learn_info",
           "mdrq_learn_window_rows", "mdrq_server_start", "mdrq_server_submit", "mdrq_server_wait",
           "mdrq_server_release", "mdrq_server_stats", "mdrq_server_stop", "mdrq_prepare_batch",
           "mdrq_prepared_launch", "mdrq_prepared_wait", "mdrq_prepared_kernels", "mdrq_prepared_free",
           "mdrq_set_shared_config", "mdrq_set_shared_bits_budget", "mdrq_autotune",
           "mdrq_set_zone_maps", "mdrq_zone_map_info", "mdrq_zone_scan_info",
           "mdrq_server_submit_batch", "mdrq_server_wait_many", "mdrq_explain_query",
           "mdrq_learn_search_info", "mdrq_learn_export", "mdrq_set_host_answers", "mdrq_set_shared_codes",
           "mdrq_set_output_order",
           "mdrq_set_key_cells"]

FAULT_SKIP_TILES, FAULT_NOMEM, FAULT_STAGE_NOMEM = 1, 2, 3
BATCH_AUTO, BATCH_PLAIN, BATCH_SHARED, BATCH_LEARNED = 0, 1, 2, 3
MODEL_PLA, MODEL_MLP, MODEL_NONE = 1, 2, 3
ZONES_OFF, ZONES_AUTO, ZONES_ALL = 0, 1, 2
HOST_AUTO, HOST_STAGED, HOST_DIRECT = 0, 1, 2
ORDER_AUTO, ORDER_LOOKBACK, ORDER_STAGED = 0, 1, 2

STATIC_MAX_ROWS = 1 << 28  # MDRQ_STATIC_MAX_ROWS


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmdrq.so is not built (run __graft_entry__.build()): %s" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32
        L.mdrq_load_columns.restype = ctypes.c_int
        L.mdrq_load_columns.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(i32), u32, u64,
                                        ctypes.c_int, vp, ctypes.POINTER(vp)]
        L.mdrq_query.restype = ctypes.c_int
        L.mdrq_query.argtypes = [vp, ctypes.POINTER(Pred), u32, vp, u64,
                                 ctypes.POINTER(u64), ctypes.c_int, vp]
        L.mdrq_query_batch.restype = ctypes.c_int
        L.mdrq_query_batch.argtypes = [vp, ctypes.POINTER(QDesc), u32, vp, u64,
                                       ctypes.POINTER(u64), ctypes.c_int, vp]
        L.mdrq_free.restype = None
        L.mdrq_free.argtypes = [vp]
        L.mdrq_status_string.restype = ctypes.c_char_p
        L.mdrq_status_string.argtypes = [ctypes.c_int]
        L.mdrq_table_rows.restype = u64
        L.mdrq_table_rows.argtypes = [vp]
        L.mdrq_table_dims.restype = u32
        L.mdrq_table_dims.argtypes = [vp]
        L.mdrq_last_scan_stats.restype = None
        L.mdrq_last_scan_stats.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64)]
        L.mdrq_scan_timing.restype = ctypes.c_int
        L.mdrq_scan_timing.argtypes = [vp, ctypes.c_int]
        L.mdrq_scan_timing_read.restype = ctypes.c_int
        L.mdrq_scan_timing_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(u64),
                                            ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.c_int]
        L.mdrq_learn.restype = ctypes.c_int
        L.mdrq_learn.argtypes = [vp, ctypes.POINTER(u32), u32, ctypes.c_int, vp]
        L.mdrq_learn_info.restype = ctypes.c_int
        L.mdrq_learn_info.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u32), ctypes.POINTER(ctypes.c_double)]
        L.mdrq_learn_window_rows.restype = ctypes.c_int
        L.mdrq_learn_window_rows.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64)]
        L.mdrq_set_key_cells.restype = ctypes.c_int
        L.mdrq_set_key_cells.argtypes = [vp, u32, ctypes.POINTER(ctypes.c_float), u32]
        L.mdrq_set_shared_codes.restype = ctypes.c_int
        L.mdrq_set_shared_codes.argtypes = [vp, ctypes.c_int]
        L.mdrq_set_host_answers.restype = ctypes.c_int
        L.mdrq_set_host_answers.argtypes = [vp, ctypes.c_int]
        L.mdrq_set_output_order.restype = ctypes.c_int
        L.mdrq_set_output_order.argtypes = [vp, ctypes.c_int]
        L.mdrq_learn_export.restype = ctypes.c_int
        L.mdrq_learn_export.argtypes = [vp, ctypes.POINTER(ModelDesc), ctypes.POINTER(u64), ctypes.POINTER(u64),
                                        ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), u32]
        L.mdrq_learn_search_info.restype = ctypes.c_int
        L.mdrq_learn_search_info.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64)]
        L.mdrq_set_batch_mode.restype = ctypes.c_int
        L.mdrq_set_batch_mode.argtypes = [vp, ctypes.c_int]
        L.mdrq_server_start.restype = ctypes.c_int
        L.mdrq_server_start.argtypes = [vp, u64, u32, ctypes.POINTER(vp)]
        L.mdrq_server_submit.restype = ctypes.c_int
        L.mdrq_server_submit.argtypes = [vp, ctypes.POINTER(Pred), u32, ctypes.POINTER(u64)]
        L.mdrq_server_wait.restype = ctypes.c_int
        L.mdrq_server_wait.argtypes = [vp, u64, ctypes.c_int64, ctypes.POINTER(vp), ctypes.POINTER(u64),
                                       ctypes.POINTER(ctypes.c_double)]
        L.mdrq_server_release.restype = ctypes.c_int
        L.mdrq_server_release.argtypes = [vp, u64]
        L.mdrq_server_stats.restype = ctypes.c_int
        L.mdrq_server_stats.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(u64),
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        L.mdrq_server_stop.restype = ctypes.c_int
        L.mdrq_server_stop.argtypes = [vp]
        L.mdrq_inject_fault.restype = ctypes.c_int
        L.mdrq_inject_fault.argtypes = [vp, ctypes.c_int, u64]
        L.mdrq_query_static.restype = ctypes.c_int
        L.mdrq_query_static.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(i32), u32, u64,
                                        ctypes.POINTER(Pred), u32, vp, u64, ctypes.POINTER(u64), vp]
        L.mdrq_server_submit_batch.restype = ctypes.c_int
        L.mdrq_server_submit_batch.argtypes = [vp, ctypes.POINTER(QDesc), u32, ctypes.POINTER(u64)]
        L.mdrq_server_wait_many.restype = ctypes.c_int
        L.mdrq_server_wait_many.argtypes = [vp, ctypes.POINTER(u64), u32, ctypes.c_int64, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(u64), ctypes.POINTER(ctypes.c_double), ctypes.c_int]
        L.mdrq_set_zone_maps.restype = ctypes.c_int
        L.mdrq_set_zone_maps.argtypes = [vp, ctypes.c_int]
        L.mdrq_zone_map_info.restype = ctypes.c_int
        L.mdrq_zone_map_info.argtypes = [vp, u32, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
        L.mdrq_zone_scan_info.restype = ctypes.c_int
        L.mdrq_zone_scan_info.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64)]
        L.mdrq_set_shared_config.restype = ctypes.c_int
        L.mdrq_set_shared_config.argtypes = [vp, u32, u32]
        L.mdrq_set_shared_bits_budget.restype = ctypes.c_int
        L.mdrq_set_shared_bits_budget.argtypes = [vp, u64]
        L.mdrq_autotune.restype = ctypes.c_int
        L.mdrq_autotune.argtypes = [vp, ctypes.POINTER(QDesc), u32, vp, ctypes.POINTER(Tuning)]
        L.mdrq_prepare_batch.restype = ctypes.c_int
        L.mdrq_prepare_batch.argtypes = [vp, ctypes.POINTER(QDesc), u32, vp, u64, ctypes.POINTER(u64), vp,
                                         ctypes.POINTER(vp)]
        L.mdrq_prepared_launch.restype = ctypes.c_int
        L.mdrq_prepared_launch.argtypes = [vp, vp]
        L.mdrq_prepared_wait.restype = ctypes.c_int
        L.mdrq_prepared_wait.argtypes = [vp, ctypes.POINTER(u64), vp]
        L.mdrq_prepared_kernels.restype = ctypes.c_int
        L.mdrq_prepared_kernels.argtypes = [vp, ctypes.POINTER(u64)]
        L.mdrq_prepared_free.restype = None
        L.mdrq_prepared_free.argtypes = [vp]
        L.mdrq_explain_query.restype = ctypes.c_int
        L.mdrq_explain_query.argtypes = [vp, ctypes.POINTER(Pred), u32, ctypes.POINTER(Pred), u32,
                                         ctypes.POINTER(u32), ctypes.POINTER(ctypes.c_int)]
        _lib = L
    return _lib


def status_string(status: int) -> str:
    try:
        return lib().mdrq_status_string(int(status)).decode()
    except RuntimeError:
        return "status %d" % status


def _bits(v, dtype: int) -> int:
    if dtype == F32:
        return int(np.array([v], dtype=np.float32).view(np.uint32)[0])
    iv = int(v)
    if not -2**31 <= iv < 2**31:
        raise ValueError("int32 bound out of range: %r" % v)
    return iv & 0xFFFFFFFF


def _unbits(b: int, dtype: int):
    """Inverse of ``_bits``: a bound's bit pattern as a Python float or int."""
    if dtype == F32:
        return float(np.array([b], dtype=np.uint32).view(np.float32)[0])
    return int(np.array([b], dtype=np.uint32).view(np.int32)[0])


def encode_query(query, dtypes) -> ctypes.Array:
    """(dim, lo, hi) predicates -> a ctypes array of mdrq_pred (bounds in column type)."""
    arr = (Pred * max(1, len(query)))()
    for i, (j, lo, hi) in enumerate(query):
        j = int(j)
        if not 0 <= j < len(dtypes):
            raise ValueError("dimension %d out of range" % j)
        arr[i].dim = j
        arr[i].reserved = 0
        arr[i].lo = _bits(lo, dtypes[j])
        arr[i].hi = _bits(hi, dtypes[j])
    return arr


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def as_uint32_numpy(t) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint32)


def query_static(columns, query, out, stream=None):
    """``mdrq_query_static``: one query over caller-owned device columns with no memory
    allocated by the library (its scratch is a fixed device array). ``columns``: d
    contiguous 1-D CUDA tensors (float32 / int32); ``out``: device int32 tensor whose
    length is the capacity. Returns (status, answer length)."""
    import torch
    dtypes = []
    for c in columns:
        if not (isinstance(c, torch.Tensor) and c.is_cuda and c.dim() == 1 and c.is_contiguous()):
            raise ValueError("columns must be contiguous 1-D CUDA tensors")
        dt = {torch.float32: F32, torch.int32: I32}.get(c.dtype)
        if dt is None:
            raise TypeError("columns must be float32 or int32")
        dtypes.append(dt)
    d = len(columns)
    n = columns[0].numel() if d else 0
    preds = encode_query(query, dtypes)
    cnt = ctypes.c_uint64(0)
    st = lib().mdrq_query_static((ctypes.c_void_p * max(1, d))(*[c.data_ptr() for c in columns]),
                                 (ctypes.c_int32 * max(1, d))(*dtypes), d, n, preds, len(query),
                                 out.data_ptr(), out.numel(), ctypes.byref(cnt),
                                 _stream_handle(stream))
    return st, int(cnt.value)


class Table:
    """A table resident on the current CUDA device (``mdrq_load_columns``).

    ``columns``: d CUDA tensors (float32 / int32, 1-D, same length) referenced in place
    (they must stay alive and unchanged), or d numpy arrays copied to the device.
    """

    def __init__(self, columns, stream=None):
        import torch
        L = lib()
        if not torch.cuda.is_available():
            raise RuntimeError("MDRQ tables need a CUDA device")
        self._keep = []
        on_device = all(isinstance(c, torch.Tensor) and c.is_cuda for c in columns)
        ptrs, dtypes = [], []
        n = None
        for c in columns:
            if on_device:
                if c.dim() != 1 or not c.is_contiguous():
                    raise ValueError("device columns must be contiguous 1-D tensors")
                dt = {torch.float32: F32, torch.int32: I32}.get(c.dtype)
                ptrs.append(c.data_ptr())
                ln = c.numel()
            else:
                a = np.ascontiguousarray(c)
                dt = {np.dtype(np.float32): F32, np.dtype(np.int32): I32}.get(a.dtype)
                ptrs.append(a.ctypes.data)
                ln = a.shape[0]
                c = a
            if dt is None:
                raise TypeError("columns must be float32 or int32")
            if n is None:
                n = ln
            elif n != ln:
                raise ValueError("columns differ in length")
            dtypes.append(dt)
            self._keep.append(c)
        self.n = int(n or 0)
        self.d = len(columns)
        self.dtypes = dtypes
        h = ctypes.c_void_p()
        st = L.mdrq_load_columns((ctypes.c_void_p * max(1, self.d))(*ptrs),
                                 (ctypes.c_int32 * max(1, self.d))(*dtypes), self.d, self.n,
                                 1 if on_device else 0, _stream_handle(stream), ctypes.byref(h))
        if not on_device:
            self._keep = []  # the library holds its own copy now
        if st != OK:
            raise MDRQError(st, "mdrq_load_columns")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().mdrq_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    # ------------------------------------------------------------------ queries

    def query(self, query, out=None, stream=None):
        """Answer one query; returns a device int32 tensor of ascending ids.

        ``out``: optional preallocated device int32 tensor; its length is the capacity.
        Without it the answer is sized exactly (a count call first if needed)."""
        import torch
        preds = encode_query(query, self.dtypes)
        cnt = ctypes.c_uint64(0)
        if out is None:
            cap = min(self.n, 1 << 20)
            out = torch.empty(max(1, cap), dtype=torch.int32, device="cuda")
            st = lib().mdrq_query(self._h, preds, len(query), out.data_ptr(), cap,
                                  ctypes.byref(cnt), 1, _stream_handle(stream))
            if st == E_CAPACITY:
                out = torch.empty(int(cnt.value), dtype=torch.int32, device="cuda")
                st = lib().mdrq_query(self._h, preds, len(query), out.data_ptr(), out.numel(),
                                      ctypes.byref(cnt), 1, _stream_handle(stream))
        else:
            st = lib().mdrq_query(self._h, preds, len(query), out.data_ptr(), out.numel(),
                                  ctypes.byref(cnt), 1, _stream_handle(stream))
        if st != OK:
            raise MDRQError(st, "mdrq_query")
        return out[: int(cnt.value)]

    def explain(self, query):
        """``mdrq_explain_query``: (empty, [(dim, lo, hi), ...]) — whether the query is
        answered empty without a scan, and the predicates the scan evaluates in order,
        with bounds as Python numbers of the columns' types."""
        preds = encode_query(query, self.dtypes)
        cap = max(1, len(query))
        plan = (Pred * cap)()
        k, empty = ctypes.c_uint32(0), ctypes.c_int(0)
        st = lib().mdrq_explain_query(self._h, preds, len(query), plan, cap, ctypes.byref(k), ctypes.byref(empty))
        if st != OK:
            raise MDRQError(st, "mdrq_explain_query")
        out = []
        for i in range(int(k.value)):
            j = int(plan[i].dim)
            lo, hi = _unbits(plan[i].lo, self.dtypes[j]), _unbits(plan[i].hi, self.dtypes[j])
            out.append((j, lo, hi))
        return bool(empty.value), out

    def query_host(self, query, capacity=None, stream=None) -> np.ndarray:
        """Answer one query into host memory (``ids_on_device = 0``); uint32 numpy array."""
        preds = encode_query(query, self.dtypes)
        cap = self.n if capacity is None else int(capacity)
        out = np.empty(max(1, cap), dtype=np.uint32)
        cnt = ctypes.c_uint64(0)
        st = lib().mdrq_query(self._h, preds, len(query), out.ctypes.data, cap, ctypes.byref(cnt),
                              0, _stream_handle(stream))
        if st != OK:
            raise MDRQError(st, "mdrq_query")
        return out[: int(cnt.value)]

    def encode_batch(self, queries):
        """Pre-encode a batch (the ctypes arrays must outlive the call)."""
        keep = [encode_query(q, self.dtypes) for q in queries]
        descs = (QDesc * max(1, len(queries)))()
        for i, (q, a) in enumerate(zip(queries, keep)):
            descs[i].preds = ctypes.cast(a, ctypes.POINTER(Pred))
            descs[i].npreds = len(q)
            descs[i].reserved = 0
        return descs, keep, len(queries)

    def query_batch_raw(self, encoded, ids_ptr: int, capacity: int, ids_on_device: bool,
                        stream=None):
        """One ``mdrq_query_batch`` call; returns (status, offsets uint64 numpy)."""
        descs, _keep, nq = encoded
        offsets = np.zeros(nq + 1, dtype=np.uint64)
        st = lib().mdrq_query_batch(self._h, descs, nq, ids_ptr, int(capacity),
                                    offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                    1 if ids_on_device else 0, _stream_handle(stream))
        return st, offsets

    def query_batch(self, queries, out=None, stream=None):
        """Answer a batch; returns (device int32 ids tensor, offsets uint64 numpy)."""
        import torch
        enc = self.encode_batch(queries)
        if out is None:
            cap = min(self.n * max(1, len(queries)), 1 << 22)
            out = torch.empty(max(1, cap), dtype=torch.int32, device="cuda")
        st, off = self.query_batch_raw(enc, out.data_ptr(), out.numel(), True, stream)
        if st == E_CAPACITY:
            out = torch.empty(int(off[-1]), dtype=torch.int32, device="cuda")
            st, off = self.query_batch_raw(enc, out.data_ptr(), out.numel(), True, stream)
        if st != OK:
            raise MDRQError(st, "mdrq_query_batch")
        return out[: int(off[-1])], off

    def set_shared_codes(self, enable: bool):
        """``mdrq_set_shared_codes``: let the shared scan encode its columns (default on)."""
        st = lib().mdrq_set_shared_codes(self._h, 1 if enable else 0)
        if st != OK:
            raise MDRQError(st, "mdrq_set_shared_codes")

    def set_host_answers(self, mode: int):
        """``mdrq_set_host_answers``: HOST_AUTO, HOST_STAGED or HOST_DIRECT."""
        st = lib().mdrq_set_host_answers(self._h, int(mode))
        if st != OK:
            raise MDRQError(st, "mdrq_set_host_answers")

    def set_output_order(self, mode: int):
        """``mdrq_set_output_order``: ORDER_AUTO, ORDER_LOOKBACK or ORDER_STAGED."""
        st = lib().mdrq_set_output_order(self._h, int(mode))
        if st != OK:
            raise MDRQError(st, "mdrq_set_output_order")

    def set_zone_maps(self, mode: int):
        """``mdrq_set_zone_maps``: ZONES_OFF, ZONES_AUTO or ZONES_ALL."""
        st = lib().mdrq_set_zone_maps(self._h, int(mode))
        if st != OK:
            raise MDRQError(st, "mdrq_set_zone_maps")

    def zone_map_info(self, dim: int) -> dict:
        used, width = ctypes.c_int(0), ctypes.c_double(0)
        st = lib().mdrq_zone_map_info(self._h, int(dim), ctypes.byref(used), ctypes.byref(width))
        if st != OK:
            raise MDRQError(st, "mdrq_zone_map_info")
        return {"used": bool(used.value), "mean_width": width.value}

    def zone_scan_info(self) -> tuple:
        """(rows, tiles) the last zone-pruned launch visited."""
        r, k = ctypes.c_uint64(0), ctypes.c_uint64(0)
        st = lib().mdrq_zone_scan_info(self._h, ctypes.byref(r), ctypes.byref(k))
        if st != OK:
            raise MDRQError(st, "mdrq_zone_scan_info")
        return int(r.value), int(k.value)

    def set_shared_config(self, unit_rows: int = 0, image_kib: int = 0):
        """``mdrq_set_shared_config``: the shared scan's rows per warp unit and chunk
        shared-memory budget (0: built-in)."""
        st = lib().mdrq_set_shared_config(self._h, int(unit_rows), int(image_kib))
        if st != OK:
            raise MDRQError(st, "mdrq_set_shared_config")

    def set_shared_bits_budget(self, max_bytes: int):
        """``mdrq_set_shared_bits_budget``: device bytes the shared scan may keep for row
        query bits between its passes (0: never; ``2**64 - 1``: the default)."""
        st = lib().mdrq_set_shared_bits_budget(self._h, int(max_bytes))
        if st != OK:
            raise MDRQError(st, "mdrq_set_shared_bits_budget")

    def autotune(self, queries, stream=None) -> dict:
        """``mdrq_autotune`` on this batch; returns the ``mdrq_tuning`` fields."""
        descs, _keep, nq = self.encode_batch(queries)
        r = Tuning()
        st = lib().mdrq_autotune(self._h, descs, nq, _stream_handle(stream), ctypes.byref(r))
        if st != OK:
            raise MDRQError(st, "mdrq_autotune")
        return {k: getattr(r, k) for k, _ in Tuning._fields_}

    def prepare(self, queries, out=None, stream=None) -> "Prepared":
        """``mdrq_prepare_batch``: the batch recorded as a CUDA graph for replays. ``out``
        (device int32 tensor) receives every replay's answer; by default one of the
        exact size is made from a first run."""
        import torch
        enc = self.encode_batch(queries)
        descs, _keep, nq = enc
        off = np.zeros(nq + 1, dtype=np.uint64)
        h = ctypes.c_void_p(0)

        def attempt(buf):
            return lib().mdrq_prepare_batch(self._h, descs, nq, buf.data_ptr(), buf.numel(),
                                            off.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                            _stream_handle(stream), ctypes.byref(h))
        if out is None:
            probe = torch.empty(1, dtype=torch.int32, device="cuda")
            st = attempt(probe)
            if st == OK:
                out = probe
            elif st == E_CAPACITY:
                out = torch.empty(max(1, int(off[-1])), dtype=torch.int32, device="cuda")
                st = attempt(out)
        else:
            st = attempt(out)
        if st != OK:
            raise MDRQError(st, "mdrq_prepare_batch")
        return Prepared(self, h.value, out, nq, off.copy())

    def learn(self, dims, model: int = MODEL_PLA, stream=None, cells=None):
        """``mdrq_learn``: a learned range narrower over the Z-order key of ``dims`` (the
        rows must be sorted by that key). ``cells``: per key dimension 255 ascending
        float32 cell bounds (``mdrq_set_key_cells``), or None for equal-width cells.
        Returns ``learn_info()``."""
        for k, j in enumerate(dims):
            b = None if cells is None else cells[k]
            if b is None:
                st = lib().mdrq_set_key_cells(self._h, int(j), None, 0)
            else:
                b = np.ascontiguousarray(b, dtype=np.float32)
                st = lib().mdrq_set_key_cells(self._h, int(j), b.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                              b.size)
            if st != OK:
                raise MDRQError(st, "mdrq_set_key_cells")
        arr = (ctypes.c_uint32 * max(1, len(dims)))(*[int(j) for j in dims])
        st = lib().mdrq_learn(self._h, arr, len(dims), int(model), _stream_handle(stream))
        if st != OK:
            raise MDRQError(st, "mdrq_learn")
        return self.learn_info()

    def learn_info(self) -> dict:
        e, sg, ms = ctypes.c_uint64(0), ctypes.c_uint32(0), ctypes.c_double(0)
        st = lib().mdrq_learn_info(self._h, ctypes.byref(e), ctypes.byref(sg), ctypes.byref(ms))
        if st != OK:
            raise MDRQError(st, "mdrq_learn_info")
        return {"max_error": int(e.value), "segments": int(sg.value), "train_ms": ms.value}

    def learn_window_rows(self) -> tuple:
        """(rows the last learned batch's windows covered, widening steps taken)."""
        r, w = ctypes.c_uint64(0), ctypes.c_uint64(0)
        st = lib().mdrq_learn_window_rows(self._h, ctypes.byref(r), ctypes.byref(w))
        if st != OK:
            raise MDRQError(st, "mdrq_learn_window_rows")
        return int(r.value), int(w.value)

    def learn_search_info(self) -> tuple:
        """(key ranges searched, keys read by the searches) of the last learned batch."""
        r, k = ctypes.c_uint64(0), ctypes.c_uint64(0)
        st = lib().mdrq_learn_search_info(self._h, ctypes.byref(r), ctypes.byref(k))
        if st != OK:
            raise MDRQError(st, "mdrq_learn_search_info")
        return int(r.value), int(k.value)

    def learn_export(self) -> dict:
        """``mdrq_learn_export``: the model's description and parameters as numpy arrays."""
        d = ModelDesc()
        st = lib().mdrq_learn_export(self._h, ctypes.byref(d), None, None, None, None, 0)
        if st != OK:
            raise MDRQError(st, "mdrq_learn_export")
        cap = d.segments + 1
        kk = np.zeros(cap, dtype=np.uint64)
        kp = np.zeros(cap, dtype=np.uint64)
        sl = np.zeros(max(1, d.segments), dtype=np.float32)
        w = np.zeros(max(1, d.mlp_params), dtype=np.float32)
        P = ctypes.POINTER
        st = lib().mdrq_learn_export(self._h, ctypes.byref(d), kk.ctypes.data_as(P(ctypes.c_uint64)),
                                     kp.ctypes.data_as(P(ctypes.c_uint64)), sl.ctypes.data_as(P(ctypes.c_float)),
                                     w.ctypes.data_as(P(ctypes.c_float)), cap)
        if st != OK:
            raise MDRQError(st, "mdrq_learn_export")
        entries = d.segments + 1 if d.kind == MODEL_PLA else d.segments
        return {"kind": d.kind, "segments": d.segments, "key_min": int(d.key_min), "key_inv": np.float32(d.key_inv),
                "max_error": int(d.max_error), "knot_key": kk[:entries], "knot_pos": kp[:entries],
                "slope": sl[:d.segments], "mlp": w[:d.mlp_params]}

    def set_batch_mode(self, mode: int):
        """``mdrq_set_batch_mode``: BATCH_AUTO, BATCH_PLAIN or BATCH_SHARED."""
        st = lib().mdrq_set_batch_mode(self._h, int(mode))
        if st != OK:
            raise MDRQError(st, "mdrq_set_batch_mode")

    def inject_fault(self, kind: int, arg: int = 0):
        """Arm a test fault for the next query call (``mdrq_inject_fault``)."""
        st = lib().mdrq_inject_fault(self._h, int(kind), int(arg))
        if st != OK:
            raise MDRQError(st, "mdrq_inject_fault")

    def scan_timing(self, enable: bool):
        st = lib().mdrq_scan_timing(self._h, 1 if enable else 0)
        if st != OK:
            raise MDRQError(st, "mdrq_scan_timing")

    def scan_timing_read(self, reset: bool = True) -> dict:
        ms = ctypes.c_double(0)
        a, b, c = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
        st = lib().mdrq_scan_timing_read(self._h, ctypes.byref(ms), ctypes.byref(a), ctypes.byref(b),
                                         ctypes.byref(c), 1 if reset else 0)
        if st != OK:
            raise MDRQError(st, "mdrq_scan_timing_read")
        return {"ms": ms.value, "scan_launches": int(a.value), "bytes": int(b.value),
                "kernel_launches": int(c.value)}

    def last_scan_stats(self):
        a, b = ctypes.c_uint64(0), ctypes.c_uint64(0)
        lib().mdrq_last_scan_stats(self._h, ctypes.byref(a), ctypes.byref(b))
        return int(a.value), int(b.value)


class Prepared:
    """A prepared batch (``mdrq_prepare_batch``): ``launch()`` enqueues a replay of its
    graph, ``wait()`` returns the offsets; ``run()`` does both and returns
    (ids tensor view, offsets). The table must outlive it."""

    def __init__(self, table: "Table", handle: int, out, nq: int, first_offsets):
        self.table = table
        self._h = handle
        self.out = out
        self.nq = nq
        self.first_offsets = first_offsets

    def launch(self, stream=None):
        st = lib().mdrq_prepared_launch(self._h, _stream_handle(stream))
        if st != OK:
            raise MDRQError(st, "mdrq_prepared_launch")

    def wait(self, stream=None) -> np.ndarray:
        off = np.zeros(self.nq + 1, dtype=np.uint64)
        st = lib().mdrq_prepared_wait(self._h, off.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                      _stream_handle(stream))
        if st != OK:
            raise MDRQError(st, "mdrq_prepared_wait")
        return off

    def run(self, stream=None):
        self.launch(stream)
        off = self.wait(stream)
        return self.out[: int(off[-1])], off

    def kernels(self) -> int:
        k = ctypes.c_uint64(0)
        st = lib().mdrq_prepared_kernels(self._h, ctypes.byref(k))
        if st != OK:
            raise MDRQError(st, "mdrq_prepared_kernels")
        return int(k.value)

    def close(self):
        if self._h:
            lib().mdrq_prepared_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class _DeviceIds:
    """A device id array the library owns, seen through __cuda_array_interface__ as int32
    (the uint32 bit patterns, as the other device answers of this binding)."""

    def __init__(self, ptr: int, count: int):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": "<i4", "data": (ptr, False),
                                         "version": 3}


class Server:
    """Continuous-batching server on a table (``mdrq_server_*``).

    ``submit`` is non-blocking and thread-safe; ``wait`` returns the answer as a device
    tensor viewing the server's result arena (valid until ``release``)."""

    def __init__(self, table: "Table", result_bytes: int = 2 << 30, max_batch: int = 512):
        h = ctypes.c_void_p()
        st = lib().mdrq_server_start(table.handle, int(result_bytes), int(max_batch), ctypes.byref(h))
        if st != OK:
            raise MDRQError(st, "mdrq_server_start")
        self._h = h
        self._table = table

    def submit_encoded(self, preds, npreds: int) -> int:
        tk = ctypes.c_uint64(0)
        st = lib().mdrq_server_submit(self._h, preds, npreds, ctypes.byref(tk))
        if st != OK:
            raise MDRQError(st, "mdrq_server_submit")
        return int(tk.value)

    def submit(self, query) -> int:
        return self.submit_encoded(encode_query(query, self._table.dtypes), len(query))

    def wait(self, ticket: int, timeout_us: int = -1):
        """(status, device uint32 tensor or None, count, latency in us)."""
        import torch
        ptr, cnt, lat = ctypes.c_void_p(), ctypes.c_uint64(0), ctypes.c_double(0)
        st = lib().mdrq_server_wait(self._h, int(ticket), int(timeout_us), ctypes.byref(ptr),
                                    ctypes.byref(cnt), ctypes.byref(lat))
        ids = None
        if st == OK and cnt.value:
            ids = torch.as_tensor(_DeviceIds(int(ptr.value), int(cnt.value)), device="cuda")
        return st, ids, int(cnt.value), lat.value

    def submit_batch(self, encoded) -> np.ndarray:
        """``mdrq_server_submit_batch`` of a batch from ``Table.encode_batch``; returns the
        tickets (uint64)."""
        descs, _keep, nq = encoded
        tk = np.zeros(max(1, nq), dtype=np.uint64)
        st = lib().mdrq_server_submit_batch(self._h, descs, nq, tk.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
        if st != OK:
            raise MDRQError(st, "mdrq_server_submit_batch")
        return tk[:nq]

    def wait_many(self, tickets, release: bool = True, timeout_us: int = -1):
        """``mdrq_server_wait_many``: (status int32, counts uint64, latency_us float64)
        arrays for the tickets, answers released when ``release``."""
        tk = np.ascontiguousarray(np.asarray(tickets, dtype=np.uint64))
        n = tk.size
        status = np.zeros(max(1, n), dtype=np.int32)
        counts = np.zeros(max(1, n), dtype=np.uint64)
        lat = np.zeros(max(1, n), dtype=np.float64)
        st = lib().mdrq_server_wait_many(self._h, tk.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), n,
                                         int(timeout_us), status.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                         counts.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                         lat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1 if release else 0)
        if st != OK:
            raise MDRQError(st, "mdrq_server_wait_many")
        return status[:n], counts[:n], lat[:n]

    def release(self, ticket: int):
        st = lib().mdrq_server_release(self._h, int(ticket))
        if st != OK:
            raise MDRQError(st, "mdrq_server_release")

    def stats(self) -> dict:
        c, b, d = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
        p50, p99 = ctypes.c_double(0), ctypes.c_double(0)
        lib().mdrq_server_stats(self._h, ctypes.byref(c), ctypes.byref(b), ctypes.byref(d),
                                ctypes.byref(p50), ctypes.byref(p99))
        return {"completed": int(c.value), "batches": int(b.value), "deferred": int(d.value),
                "p50_us": p50.value, "p99_us": p99.value}

    def stop(self) -> int:
        st = OK
        if getattr(self, "_h", None):
            st = lib().mdrq_server_stop(self._h)
            self._h = None
        return st

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass
