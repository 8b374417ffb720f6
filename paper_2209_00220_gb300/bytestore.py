"""ctypes binding of libbytestore with the C ABI's names (include/bytestore.h).

Argument marshalling only: every step of a scan or lookup runs in the CUDA
library. Device buffers are torch CUDA tensors (result bit vectors are int32
tensors holding uint32 words); streams default to torch's current stream.
The library is loaded on first use; if it is missing this module raises
ImportError -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbytestore.so")

LAYOUTS = {"bitpacked": 0, "byteslice": 1, "ppvbs": 2}
OPS = {"lt": 0, "le": 1, "gt": 2, "ge": 3, "eq": 4, "ne": 5, "between": 6}
ADVISE_TIMED, ADVISE_BYTES_MODEL = 0, 1

BS_OK, BS_ERR_INVALID_ARG, BS_ERR_OOM, BS_ERR_CUDA = 0, -1, -2, -3
BS_ERR_CAPACITY, BS_ERR_UNSUPPORTED, BS_ERR_TIMEOUT, BS_ERR_DEVICE_CHECK, BS_ERR_NOT_READY = -4, -5, -6, -7, -8

_u64, _i32, _i64, _vp = ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p


class bs_encode_opts(ctypes.Structure):
    _fields_ = [("domain_bits", _i32), ("device", _i32), ("domain_min", _i64), ("domain_values", _vp),
                ("n_domain", _u64), ("host_only", _i32), ("keep_host", _i32), ("threads", _i32),
                ("categorical", _i32), ("domain_counts", _vp)]


class bs_column_info(ctypes.Structure):
    _fields_ = [("n_rows", _u64), ("layout", _i32), ("max_code_bytes", _i32), ("code_bits", _i32),
                ("on_device", _i32), ("n_dict", _u64), ("device_bytes", _u64), ("layout_bytes", _u64),
                ("len_hist", _u64 * 9)]


class bs_pred(ctypes.Structure):
    _fields_ = [("col", _vp), ("op", _i32), ("lit", _i32), ("lit2", _i32), ("reserved", _i32)]


class bs_scan_bytes_t(ctypes.Structure):
    _fields_ = [("bytes", _u64), ("dense_bytes", _u64), ("mask_bytes", _u64), ("offset_bytes", _u64),
                ("deep_bytes", _u64), ("result_bytes", _u64), ("paper_model_bytes", _u64),
                ("pending_rows", _u64 * 9), ("sampled_tiles", _u64)]


class bs_lookup_bytes_t(ctypes.Structure):
    _fields_ = [("bytes", _u64), ("selected", _u64), ("bits_bytes", _u64), ("out_bytes", _u64),
                ("dense_bytes", _u64), ("mask_bytes", _u64), ("offset_bytes", _u64), ("deep_bytes", _u64)]


class bs_request(ctypes.Structure):
    _fields_ = [("npreds", _i32), ("reserved", _i32), ("preds", bs_pred * 4), ("proj", _vp), ("d_out", _vp),
                ("out_cap", _u64), ("d_count", _vp), ("d_bits", _vp)]


class bs_batch_opts(ctypes.Structure):
    _fields_ = [("threads", _i32), ("blocks_per_sm", _i32), ("autotune", _i32), ("use_graph", _i32),
                ("tune_cache", ctypes.c_char_p), ("stages", _i32), ("unit_chunks", _i32), ("stop_rows", _i32),
                ("reserved", _i32)]


class bs_batch_shape(ctypes.Structure):
    _fields_ = [("threads", _i32), ("blocks_per_sm", _i32), ("ctas", _i32), ("stages", _i32),
                ("unit_chunks", _i32), ("stop_rows", _i32), ("graph", _i32), ("persistent_requests", _i32),
                ("single_query_requests", _i32)]


class bs_query(ctypes.Structure):
    _fields_ = [("npreds", _i32), ("reserved", _i32), ("preds", bs_pred * 4), ("proj", _vp)]


class bs_server_opts(ctypes.Structure):
    _fields_ = [("max_batch", _i32), ("slots", _i32), ("result_bytes", _u64), ("scratch_bytes", _u64),
                ("threads", _i32), ("device", _i32), ("single_query_kernels", _i32), ("reserved", _i32)]


class bs_query_result(ctypes.Structure):
    _fields_ = [("status", _i32), ("reserved", _i32), ("count", _u64), ("d_values", _vp),
                ("queue_us", ctypes.c_double), ("latency_us", ctypes.c_double)]


class bs_server_stats(ctypes.Structure):
    _fields_ = [("submitted", _u64), ("completed", _u64), ("rejected", _u64), ("batches", _u64),
                ("mean_batch", ctypes.c_double), ("result_bytes_in_use", _u64), ("scratch_bytes_in_use", _u64),
                ("queued", _u64), ("failed", _u64), ("persistent_queries", _u64), ("single_query_queries", _u64)]


class bs_advice(ctypes.Structure):
    _fields_ = [("layout", _i32), ("n_points", _i32), ("auc_byteslice", ctypes.c_double),
                ("auc_ppvbs", ctypes.c_double), ("selectivity", ctypes.c_double * 100),
                ("cost_byteslice", ctypes.c_double * 100), ("cost_ppvbs", ctypes.c_double * 100)]


_SIGS = {
    "bs_encode_column": ([_vp, _u64, _i32, _vp, _vp], _i32),
    "bs_column_from_codes": ([_vp, _vp, _u64, _i32, _i32, _vp, _vp], _i32),
    "bs_column_free": ([_vp], None),
    "bs_column_get_info": ([_vp, _vp], _i32),
    "bs_column_row_codes": ([_vp, _u64, _u64, _vp, _vp], _i32),
    "bs_column_dictionary": ([_vp, _vp, _vp, _vp, _u64], _i32),
    "bs_scan": ([_vp, _i32, _i32, _i32, _vp, _vp], _i32),
    "bs_scan_seeded": ([_vp, _i32, _i32, _i32, _vp, _vp, _vp], _i32),
    "bs_scan_code": ([_vp, _i32, _u64, _i32, _u64, _i32, _vp, _vp, _vp], _i32),
    "bs_scan_conj": ([_vp, _i32, _vp, _vp], _i32),
    "bs_lookup_workspace_bytes": ([_vp], _u64),
    "bs_lookup": ([_vp, _vp, _vp, _u64, _vp, _vp, _u64, _vp], _i32),
    "bs_lookup_codes": ([_vp, _vp, _vp, _u64, _vp, _vp, _u64, _vp], _i32),
    "bs_lookup_noalloc": ([_vp, _vp, _vp, _u64, _vp, _vp], _i32),
    "bs_lookup_rowids": ([_vp, _vp, _u64, _vp, _vp], _i32),
    "bs_lookup_shape": ([_vp, _vp, _vp, _vp], _i32),
    "bs_scan_lookup_workspace_bytes": ([_vp], _u64),
    "bs_scan_lookup": ([_vp, _i32, _vp, _vp, _vp, _u64, _vp, _vp, _u64, _vp], _i32),
    "bs_advise_layout": ([_vp, _u64, _i32, _vp, _vp], _i32),
    "bs_advise_layout_range": ([_vp, _u64, _i32, _vp, ctypes.c_double, ctypes.c_double, _vp], _i32),
    "bs_selftest_bounded_wait": ([ctypes.c_uint32, _vp], _i32),
    "bs_column_save": ([_vp, ctypes.c_char_p], _i32),
    "bs_column_load": ([ctypes.c_char_p, _vp, _vp], _i32),
    "bs_scan_bytes": ([_vp, _i32, _i32, _i32, _vp, _vp], _i32),
    "bs_lookup_bytes": ([_vp, _vp, _vp], _i32),
    "bs_scan_lookup_bytes": ([_vp, _i32, _i32, _i32, _vp, _i32, _vp], _i32),
    "bs_scan_bytes_sampled": ([_vp, _i32, _i32, _i32, _vp, _u64, _vp], _i32),
    "bs_batch_create": ([_vp, _i32, _vp, _vp], _i32),
    "bs_batch_launch": ([_vp, _vp], _i32),
    "bs_batch_info": ([_vp, _vp, _vp, _vp], _i32),
    "bs_batch_free": ([_vp], None),
    "bs_batch_get_shape": ([_vp, _vp], _i32),
    "bs_estimate_rows": ([_vp, _i32, _i32, _i32, _vp], _i32),
    "bs_server_create": ([_vp, _vp], _i32),
    "bs_server_submit": ([_vp, _vp, _vp], _i32),
    "bs_server_poll": ([_vp, _u64, _vp], _i32),
    "bs_server_wait": ([_vp, _u64, _i32, _vp], _i32),
    "bs_server_release": ([_vp, _u64], _i32),
    "bs_server_copy_result": ([_vp, _u64, _vp, _u64, _vp, _vp], _i32),
    "bs_server_get_stats": ([_vp, _vp], _i32),
    "bs_server_destroy": ([_vp], None),
    "bs_server_fail_next_launches": ([_vp, _i32], _i32),
    "bs_strerror": ([_i32], ctypes.c_char_p),
    "bs_last_device_error": ([], _i32),
    "bs_version": ([], ctypes.c_char_p),
}

_lib = None
_lock = threading.Lock()


def build_library(force: bool = False) -> str:
    from . import build_lib
    return build_lib.build(force=force)


def lib():
    """The loaded libbytestore (ImportError if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError("libbytestore.so is not built (%s); run "
                                  "`python -m paper_2209_00220_gb300.build_lib`" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


class BsError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = lib().bs_strerror(status).decode()
        super().__init__("%s: %s (%d)" % (what, msg, status) if what else "%s (%d)" % (msg, status))


def _check(rc: int, what: str):
    if rc != BS_OK:
        raise BsError(rc, what)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(t):
    return None if t is None else t.data_ptr()


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _opts(domain_bits=0, domain_min=0, domain_values=None, device=-1, host_only=False, keep_host=False,
          threads=0, domain_counts=None, categorical=False):
    o = bs_encode_opts()
    o.categorical = 1 if categorical else 0
    o.domain_bits = int(domain_bits)
    o.domain_min = int(domain_min)
    o.device = int(device)
    o.host_only = 1 if host_only else 0
    o.keep_host = 1 if keep_host else 0
    o.threads = int(threads)
    keep = []
    if domain_values is not None:
        dv = _np(domain_values, np.int32)
        keep.append(dv)
        o.domain_values = dv.ctypes.data
        o.n_domain = dv.size
        if domain_counts is not None:
            dc = _np(domain_counts, np.uint64)
            if dc.size != dv.size:
                raise ValueError("domain_counts needs one count per domain value")
            keep.append(dc)
            o.domain_counts = dc.ctypes.data
    elif domain_counts is not None:
        raise ValueError("domain_counts needs domain_values")
    return o, keep


class Column:
    """Owns one bs_column (freed with the object)."""

    def __init__(self, handle: int, n: int):
        self.handle = handle
        self.n = n

    @property
    def n_words(self) -> int:
        return (self.n + 31) // 32

    def info(self) -> dict:
        return bs_column_get_info(self)

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.bs_column_free(h)

    def free(self):
        self.__del__()


# ----------------------------------------------------------------- columns
def bs_encode_column(values, layout: str = "ppvbs", **opts) -> Column:
    v = _np(values, np.int32)
    o, keep = _opts(**opts)
    out = _vp()
    _check(lib().bs_encode_column(v.ctypes.data if v.size else None, v.size, LAYOUTS[layout],
                                  ctypes.byref(o), ctypes.byref(out)), "bs_encode_column")
    del keep
    return Column(out.value, v.size)


def bs_column_from_codes(codes, lens, layout: str = "ppvbs", code_bits: int = 0, **opts) -> Column:
    c = _np(codes, np.uint64)
    ln = _np(lens, np.uint8) if lens is not None else None
    o, keep = _opts(**opts)
    out = _vp()
    _check(lib().bs_column_from_codes(c.ctypes.data if c.size else None,
                                      ln.ctypes.data if ln is not None and ln.size else None, c.size,
                                      LAYOUTS[layout], int(code_bits), ctypes.byref(o), ctypes.byref(out)),
           "bs_column_from_codes")
    return Column(out.value, c.size)


def bs_column_free(col: Column):
    col.free()


def bs_column_get_info(col: Column) -> dict:
    i = bs_column_info()
    _check(lib().bs_column_get_info(col.handle, ctypes.byref(i)), "bs_column_get_info")
    return {"n_rows": i.n_rows, "layout": i.layout, "max_code_bytes": i.max_code_bytes,
            "code_bits": i.code_bits, "on_device": bool(i.on_device), "n_dict": i.n_dict,
            "device_bytes": i.device_bytes, "layout_bytes": i.layout_bytes, "len_hist": list(i.len_hist)}


def bs_column_save(col: Column, path: str):
    _check(lib().bs_column_save(col.handle, os.fsencode(path)), "bs_column_save")


def bs_column_load(path: str, **opts) -> Column:
    """opts: device, host_only, keep_host (as for bs_encode_column)."""
    o, keep = _opts(**opts)
    out = _vp()
    _check(lib().bs_column_load(os.fsencode(path), ctypes.byref(o), ctypes.byref(out)), "bs_column_load")
    col = Column(out.value, 0)
    col.n = col.info()["n_rows"]
    return col


def bs_column_row_codes(col: Column, begin: int = 0, count: int | None = None):
    count = col.n - begin if count is None else count
    codes = np.zeros(max(1, count), np.uint64)
    lens = np.zeros(max(1, count), np.uint8)
    _check(lib().bs_column_row_codes(col.handle, begin, count, codes.ctypes.data, lens.ctypes.data),
           "bs_column_row_codes")
    return codes[:count], lens[:count]


def bs_column_dictionary(col: Column):
    nd = col.info()["n_dict"]
    v = np.zeros(max(1, nd), np.int32)
    c = np.zeros(max(1, nd), np.uint64)
    ln = np.zeros(max(1, nd), np.uint8)
    _check(lib().bs_column_dictionary(col.handle, v.ctypes.data, c.ctypes.data, ln.ctypes.data, nd),
           "bs_column_dictionary")
    return v[:nd], c[:nd], ln[:nd]


# -------------------------------------------------------------------- scan
def _bits_out(col: Column, out):
    if out is None:
        import torch
        out = torch.empty(max(1, col.n_words), dtype=torch.int32, device="cuda")
    return out


def bs_scan(col: Column, op: str, lit: int, lit2: int = 0, out=None, stream=None):
    out = _bits_out(col, out)
    _check(lib().bs_scan(col.handle, OPS[op], int(lit), int(lit2), _dptr(out), _stream(stream)), "bs_scan")
    return out


def bs_scan_seeded(col: Column, op: str, lit: int, lit2: int, seed, out=None, stream=None):
    out = _bits_out(col, out)
    _check(lib().bs_scan_seeded(col.handle, OPS[op], int(lit), int(lit2), _dptr(seed), _dptr(out),
                                _stream(stream)), "bs_scan_seeded")
    return out


def bs_scan_code(col: Column, op: str, code: int, length: int = 0, code2: int = 0, length2: int = 0,
                 seed=None, out=None, stream=None):
    out = _bits_out(col, out)
    _check(lib().bs_scan_code(col.handle, OPS[op], int(code), int(length), int(code2), int(length2),
                              _dptr(seed), _dptr(out), _stream(stream)), "bs_scan_code")
    return out


def bs_scan_conj(preds, out=None, stream=None):
    """preds: sequence of (Column, op, lit[, lit2])."""
    arr = (bs_pred * len(preds))()
    for i, p in enumerate(preds):
        arr[i].col = p[0].handle
        arr[i].op = OPS[p[1]]
        arr[i].lit = int(p[2])
        arr[i].lit2 = int(p[3]) if len(p) > 3 else 0
    out = _bits_out(preds[0][0], out)
    _check(lib().bs_scan_conj(arr, len(preds), _dptr(out), _stream(stream)), "bs_scan_conj")
    return out


# ------------------------------------------------------------------ lookup
def bs_lookup_workspace_bytes(col: Column) -> int:
    return int(lib().bs_lookup_workspace_bytes(col.handle))


def bs_lookup(col: Column, bits, out=None, out_cap: int | None = None, count=None, workspace=None,
              stream=None):
    """Returns (values tensor, count tensor (int64, 1 element on the device))."""
    import torch
    if out is None:
        out = torch.empty(max(1, col.n if out_cap is None else out_cap), dtype=torch.int32, device="cuda")
    cap = out.numel() if out_cap is None else int(out_cap)
    if count is None:
        count = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(lib().bs_lookup(col.handle, _dptr(bits), _dptr(out), cap, _dptr(count), _dptr(workspace), ws_bytes,
                           _stream(stream)), "bs_lookup")
    return out, count


def bs_lookup_noalloc(col: Column, bits, out=None, out_cap: int | None = None, count=None, stream=None):
    """bs_lookup without any allocation inside the library (its scratch is a
    fixed device array shared by all calls: serialise overlapping calls)."""
    import torch
    if out is None:
        out = torch.empty(max(1, col.n if out_cap is None else out_cap), dtype=torch.int32, device="cuda")
    cap = out.numel() if out_cap is None else int(out_cap)
    if count is None:
        count = torch.zeros(1, dtype=torch.int64, device="cuda")
    _check(lib().bs_lookup_noalloc(col.handle, _dptr(bits), _dptr(out), cap, _dptr(count), _stream(stream)),
           "bs_lookup_noalloc")
    return out, count


def bs_scan_lookup_workspace_bytes(proj: Column) -> int:
    return int(lib().bs_scan_lookup_workspace_bytes(proj.handle))


def bs_scan_lookup(preds, proj: Column | None = None, out=None, out_cap: int | None = None, count=None,
                   bits=None, workspace=None, stream=None):
    """Fused conjunction + lookup: preds [(Column, op, lit[, lit2]), ...] (1..4),
    then the values of proj (default: the first predicate's column) at the
    selected rows. bits: optional int32 tensor of ceil(n/32) words that also
    receives the result bit vector. Returns (values tensor, count tensor)."""
    import torch
    if not 1 <= len(preds) <= 4:
        raise BsError(BS_ERR_INVALID_ARG, "bs_scan_lookup: 1..4 predicates")
    arr = (bs_pred * len(preds))()
    for i, p in enumerate(preds):
        arr[i].col = p[0].handle
        arr[i].op = OPS[p[1]]
        arr[i].lit = int(p[2])
        arr[i].lit2 = int(p[3]) if len(p) > 3 else 0
    pc = proj if proj is not None else preds[0][0]
    if out is None:
        out = torch.empty(max(1, pc.n if out_cap is None else out_cap), dtype=torch.int32, device="cuda")
    cap = out.numel() if out_cap is None else int(out_cap)
    if count is None:
        count = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(lib().bs_scan_lookup(arr, len(preds), pc.handle, _dptr(bits), _dptr(out), cap, _dptr(count),
                                _dptr(workspace), ws_bytes, _stream(stream)), "bs_scan_lookup")
    return out, count


def bs_lookup_shape(col: Column) -> dict:
    """Launch shape of bs_lookup's gather kernel for this column: parts (warps
    per 16-tile chunk), grid, resident_ctas."""
    p, g, r = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().bs_lookup_shape(col.handle, ctypes.byref(p), ctypes.byref(g), ctypes.byref(r)), "bs_lookup_shape")
    return {"parts": p.value, "grid": g.value, "resident_ctas": r.value}


def bs_lookup_codes(col: Column, bits, out=None, out_cap: int | None = None, count=None, workspace=None,
                    stream=None):
    import torch
    if out is None:
        out = torch.empty(max(1, col.n if out_cap is None else out_cap), dtype=torch.int64, device="cuda")
    cap = out.numel() if out_cap is None else int(out_cap)
    if count is None:
        count = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(lib().bs_lookup_codes(col.handle, _dptr(bits), _dptr(out), cap, _dptr(count), _dptr(workspace),
                                 ws_bytes, _stream(stream)), "bs_lookup_codes")
    return out, count


def bs_lookup_rowids(col: Column, rowids, out=None, stream=None):
    import torch
    if out is None:
        out = torch.empty(max(1, rowids.numel()), dtype=torch.int32, device="cuda")
    _check(lib().bs_lookup_rowids(col.handle, _dptr(rowids), rowids.numel(), _dptr(out), _stream(stream)),
           "bs_lookup_rowids")
    return out


# ------------------------------------------------- effective-bytes counter
def _struct_dict(st) -> dict:
    out = {}
    for name, _ in st._fields_:
        v = getattr(st, name)
        out[name] = list(v) if hasattr(v, "__len__") else int(v)
    return out


def bs_scan_bytes(col: Column, op: str, lit: int, lit2: int = 0, seed=None, stride: int = 1) -> dict:
    """Bytes the scan must move at the kernels' granularity (host replay).
    seed: optional host numpy uint32 bit vector; stride > 1 replays every
    stride-th tile and scales up."""
    r = bs_scan_bytes_t()
    sd = None if seed is None else _np(seed, np.uint32)
    sp = None if sd is None else sd.ctypes.data
    if stride == 1:
        _check(lib().bs_scan_bytes(col.handle, OPS[op], int(lit), int(lit2), sp, ctypes.byref(r)), "bs_scan_bytes")
    else:
        _check(lib().bs_scan_bytes_sampled(col.handle, OPS[op], int(lit), int(lit2), sp, int(stride),
                                           ctypes.byref(r)), "bs_scan_bytes_sampled")
    return _struct_dict(r)


def bs_lookup_bytes(col: Column, bits) -> dict:
    """bits: host numpy uint32 bit vector."""
    r = bs_lookup_bytes_t()
    b = _np(bits, np.uint32)
    _check(lib().bs_lookup_bytes(col.handle, b.ctypes.data if b.size else None, ctypes.byref(r)),
           "bs_lookup_bytes")
    return _struct_dict(r)


def bs_scan_lookup_bytes(col: Column, op: str, lit: int, lit2: int, sel, write_bits: bool = True) -> dict:
    """Bytes the fused scan + lookup must move for one predicate projected onto
    its own column; sel: host numpy uint32 result bit vector."""
    r = bs_scan_bytes_t()
    b = _np(sel, np.uint32)
    _check(lib().bs_scan_lookup_bytes(col.handle, OPS[op], int(lit), int(lit2), b.ctypes.data if b.size else None,
                                      1 if write_bits else 0, ctypes.byref(r)), "bs_scan_lookup_bytes")
    return _struct_dict(r)


# ----------------------------------------------------------------- batches
class Batch:
    """A prepared batch (bs_batch): many conjunction + lookup requests run by one
    persistent launch. Keeps the request columns and output tensors alive."""

    def __init__(self, handle: int, keep):
        self.handle = handle
        self._keep = keep

    def launch(self, stream=None):
        _check(lib().bs_batch_launch(self.handle, _stream(stream)), "bs_batch_launch")

    def info(self) -> dict:
        t, c, g = _i32(), _i32(), _i32()
        _check(lib().bs_batch_info(self.handle, ctypes.byref(t), ctypes.byref(c), ctypes.byref(g)), "bs_batch_info")
        return {"threads": t.value, "ctas": c.value, "graph": bool(g.value)}

    def shape(self) -> dict:
        """The full launch shape: threads, blocks_per_sm, ctas, stages,
        unit_chunks, stop_rows, graph, persistent_requests, single_query_requests."""
        s = bs_batch_shape()
        _check(lib().bs_batch_get_shape(self.handle, ctypes.byref(s)), "bs_batch_get_shape")
        return {name: getattr(s, name) for name, _ in s._fields_}

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.bs_batch_free(h)

    def free(self):
        self.__del__()


def bs_batch_create(requests, threads: int = 0, blocks_per_sm: int = 0, autotune: bool = False,
                    use_graph: bool = True, tune_cache: str | None = None, stages: int = 0, unit_chunks: int = 0,
                    stop_rows: int = 0) -> Batch:
    """requests: sequence of dicts with keys
         preds: [(Column, op, lit[, lit2]), ...]  (1..4, equal-length columns)
         out:   torch int32 CUDA tensor (capacity = its numel unless out_cap given)
         count: torch int64 CUDA tensor of 1 element (optional)
         proj:  Column looked up (optional, default preds[0]'s column)
         bits:  torch int32 CUDA tensor receiving the bit vector (optional)"""
    arr = (bs_request * len(requests))()
    keep = []
    for i, q in enumerate(requests):
        preds = q["preds"]
        if not 1 <= len(preds) <= len(arr[i].preds):
            raise BsError(BS_ERR_INVALID_ARG, "bs_batch_create: 1..%d predicates per request" % len(arr[i].preds))
        arr[i].npreds = len(preds)
        for j, p in enumerate(preds):
            arr[i].preds[j].col = p[0].handle
            arr[i].preds[j].op = OPS[p[1]]
            arr[i].preds[j].lit = int(p[2])
            arr[i].preds[j].lit2 = int(p[3]) if len(p) > 3 else 0
            keep.append(p[0])
        proj = q.get("proj")
        arr[i].proj = proj.handle if proj is not None else None
        out = q.get("out")
        arr[i].d_out = _dptr(out)
        arr[i].out_cap = int(q.get("out_cap", out.numel() if out is not None else 0))
        arr[i].d_count = _dptr(q.get("count"))
        arr[i].d_bits = _dptr(q.get("bits"))
        keep.extend([proj, out, q.get("count"), q.get("bits")])
    o = bs_batch_opts()
    o.threads, o.blocks_per_sm = int(threads), int(blocks_per_sm)
    o.autotune, o.use_graph = 1 if autotune else 0, 1 if use_graph else 0
    o.tune_cache = tune_cache.encode() if tune_cache else None
    o.stages, o.unit_chunks, o.stop_rows = int(stages), int(unit_chunks), int(stop_rows)
    h = _vp()
    _check(lib().bs_batch_create(arr, len(requests), ctypes.byref(o), ctypes.byref(h)), "bs_batch_create")
    return Batch(h.value, keep)


def bs_batch_launch(batch: Batch, stream=None):
    batch.launch(stream)


def bs_batch_free(batch: Batch):
    batch.free()


# ----------------------------------------------------------------- serving
def bs_estimate_rows(col: Column, op: str, lit: int, lit2: int = 0) -> int:
    out = _u64()
    _check(lib().bs_estimate_rows(col.handle, OPS[op], int(lit), int(lit2), ctypes.byref(out)), "bs_estimate_rows")
    return out.value


class Server:
    """bs_server: continuous batching over resident columns."""

    def __init__(self, handle: int):
        self.handle = handle
        self._cols = []

    @staticmethod
    def prepare(preds, proj=None) -> bs_query:
        """The bs_query for (preds, proj), built ahead of submission."""
        q = bs_query()
        if not 1 <= len(preds) <= len(q.preds):
            raise BsError(BS_ERR_INVALID_ARG, "bs_server_submit: 1..%d predicates per query" % len(q.preds))
        q.npreds = len(preds)
        for j, p in enumerate(preds):
            q.preds[j].col = p[0].handle
            q.preds[j].op = OPS[p[1]]
            q.preds[j].lit = int(p[2])
            q.preds[j].lit2 = int(p[3]) if len(p) > 3 else 0
        q.proj = proj.handle if proj is not None else None
        return q

    def submit(self, preds, proj=None) -> int:
        """preds: [(Column, op, lit[, lit2]), ...], or a bs_query from prepare()."""
        q = preds if isinstance(preds, bs_query) else self.prepare(preds, proj)
        t = _u64()
        _check(lib().bs_server_submit(self.handle, ctypes.byref(q), ctypes.byref(t)), "bs_server_submit")
        return t.value

    def _res(self, r: bs_query_result) -> dict:
        return {"status": r.status, "count": r.count, "d_values": r.d_values, "queue_us": r.queue_us,
                "latency_us": r.latency_us}

    def poll(self, ticket: int):
        """None while the query runs; then a dict whose 'status' is the
        query's own (BS_OK or the error that failed it)."""
        r = bs_query_result()
        rc = lib().bs_server_poll(self.handle, ticket, ctypes.byref(r))
        if rc == BS_ERR_NOT_READY:
            return None
        if rc != BS_OK and rc == r.status:
            return self._res(r)  # the query finished with an error of its own
        _check(rc, "bs_server_poll")
        return self._res(r)

    def wait(self, ticket: int, timeout_ms: int = 60000) -> dict:
        r = bs_query_result()
        rc = lib().bs_server_wait(self.handle, ticket, int(timeout_ms), ctypes.byref(r))
        if rc != BS_OK and rc == r.status:
            return self._res(r)  # the query finished with an error of its own
        _check(rc, "bs_server_wait")
        return self._res(r)

    def fail_next_launches(self, n: int):
        """Test hook: the next n batch launches fail on the host (BS_ERR_CUDA)."""
        _check(lib().bs_server_fail_next_launches(self.handle, int(n)), "bs_server_fail_next_launches")

    def values(self, ticket: int, count: int, stream=None):
        """Copy a finished query's values into a new CUDA int32 tensor."""
        import torch
        out = torch.empty(max(1, int(count)), dtype=torch.int32, device="cuda")
        got = _u64()
        _check(lib().bs_server_copy_result(self.handle, ticket, _dptr(out), int(count), ctypes.byref(got),
                                           _stream(stream)), "bs_server_copy_result")
        return out[: got.value]

    def release(self, ticket: int):
        _check(lib().bs_server_release(self.handle, ticket), "bs_server_release")

    def stats(self) -> dict:
        st = bs_server_stats()
        _check(lib().bs_server_get_stats(self.handle, ctypes.byref(st)), "bs_server_get_stats")
        return {name: getattr(st, name) for name, _ in st._fields_}

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.bs_server_destroy(h)

    def destroy(self):
        self.__del__()


def bs_server_create(max_batch: int = 0, slots: int = 0, result_bytes: int = 0, scratch_bytes: int = 0,
                     threads: int = 0, device: int = -1, single_query_kernels: bool = False) -> Server:
    o = bs_server_opts()
    o.max_batch, o.slots, o.result_bytes, o.scratch_bytes = max_batch, slots, result_bytes, scratch_bytes
    o.threads, o.device = threads, device
    o.single_query_kernels = 1 if single_query_kernels else 0
    h = _vp()
    _check(lib().bs_server_create(ctypes.byref(o), ctypes.byref(h)), "bs_server_create")
    return Server(h.value)


# ----------------------------------------------------------------- advisor
def bs_advise_layout(values, mode: int = ADVISE_BYTES_MODEL, sel_range=None, **opts) -> dict:
    """sel_range: optional (lo, hi) selectivity range the predicates are known to fall in."""
    v = _np(values, np.int32)
    o, keep = _opts(**opts)
    a = bs_advice()
    lo, hi = (0.0, 1.0) if sel_range is None else (float(sel_range[0]), float(sel_range[1]))
    _check(lib().bs_advise_layout_range(v.ctypes.data if v.size else None, v.size, int(mode), ctypes.byref(o),
                                        lo, hi, ctypes.byref(a)), "bs_advise_layout_range")
    k = a.n_points
    return {"layout": {0: "bitpacked", 1: "byteslice", 2: "ppvbs"}[a.layout], "auc_byteslice": a.auc_byteslice,
            "auc_ppvbs": a.auc_ppvbs, "selectivity": list(a.selectivity[:k]),
            "cost_byteslice": list(a.cost_byteslice[:k]), "cost_ppvbs": list(a.cost_ppvbs[:k])}


# ------------------------------------------------------------- diagnostics
def bs_strerror(status: int) -> str:
    return lib().bs_strerror(int(status)).decode()


def bs_last_device_error() -> int:
    return int(lib().bs_last_device_error())


def bs_selftest_bounded_wait(max_polls: int = 1 << 14) -> bool:
    """True when a device wait on a flag nothing sets gave up after max_polls polls."""
    g = _i32()
    _check(lib().bs_selftest_bounded_wait(int(max_polls), ctypes.byref(g)), "bs_selftest_bounded_wait")
    return bool(g.value)


def bs_version() -> str:
    return lib().bs_version().decode()
