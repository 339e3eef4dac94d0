"""Exact k-NN similarity search over iSAX-summarised data series on one GB300 GPU.

A thin ctypes binding of the C ABI in include/msi.h: every function below has the
name of the C entry point it calls and only marshals arguments (numpy arrays and
host/device torch tensors to raw pointers, torch streams to cudaStream_t). All the
computation runs in the CUDA library libmsi.so; importing this module fails loudly
if that library has not been built (there is no CPU fallback).
"""
import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "MsiError", "Index", "msi_build", "msi_knn", "msi_knn_ex", "msi_free", "msi_status_str", "msi_last_error",
    "msi_abi_version", "msi_index_info_get", "msi_index_export", "msi_lower_bounds",
    "msi_query_stats_get", "msi_set_timing", "msi_lower_bounds_noalloc", "msi_merge_topk", "msi_schedule_get", "msi_schedule_set", "Server", "MSI_BUILD_BORROW", "MSI_BUILD_BALANCED_SPLIT", "MSI_MAX_K", "library_path",
]

MSI_OK, MSI_EINVAL, MSI_ENOMEM, MSI_ECUDA, MSI_ETIMEOUT, MSI_EINTERNAL = range(6)
MSI_BUILD_BORROW = 0x1
MSI_BUILD_BALANCED_SPLIT = 0x2
MSI_BUILD_NO_FINE_BOUND = 0x4
MSI_MAX_K = 1024
MSI_MAX_LEN = 4096


def library_path():
    return _build.LIB


if not os.path.exists(_build.LIB):
    raise ImportError(f"{_build.LIB} is missing: the CUDA library must be built first "
                      "(python -c 'import __graft_entry__ as g; g.build()')")

_lib = ctypes.CDLL(_build.LIB)


class _BuildOpts(ctypes.Structure):
    _fields_ = [("leaf_capacity", ctypes.c_int32), ("flags", ctypes.c_uint32), ("stream", ctypes.c_void_p),
                ("query_slots", ctypes.c_int32), ("slot_capacity", ctypes.c_int32)]


class _IndexInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("len", ctypes.c_int32), ("segments", ctypes.c_int32),
                ("cardinality", ctypes.c_int32), ("leaf_capacity", ctypes.c_int32), ("leaves", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("flags", ctypes.c_uint32), ("device", ctypes.c_int32),
                ("fine_segments", ctypes.c_int32)]


class _Export(ctypes.Structure):
    _fields_ = [(f, ctypes.c_void_p) for f in ("words", "perm", "leaf_begin", "env_lo", "env_hi", "thresholds", "znorm",
                                                "fine")]


class _QueryStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in (
        "queries", "leaves_total", "leaves_survived", "blocks_examined", "series_lower_bounded",
        "series_refined", "seed_series", "candidates", "rechecked", "refine_launches")] + [
        ("refine_ms", ctypes.c_double), ("filter_ms", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
        ("survivors", ctypes.c_int64), ("fine_bounded", ctypes.c_int64), ("front_fine_bounded", ctypes.c_int64),
        ("overflow_reruns", ctypes.c_int64), ("tc_pairs", ctypes.c_int64)]


_vp, _i32, _i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
_lib.msi_build.argtypes = [_vp, _i64, _i32, _i32, _i32, ctypes.POINTER(_BuildOpts), ctypes.POINTER(_vp)]
_lib.msi_build.restype = ctypes.c_int
_lib.msi_knn.argtypes = [_vp, _vp, _i64, _i32, _vp, _vp, _vp]
_lib.msi_autotune.argtypes = [_vp, _vp, _i64, _i32, _i32, _vp, _vp]
_lib.msi_autotune.restype = ctypes.c_int
_lib.msi_knn.restype = ctypes.c_int
_lib.msi_knn_ex.argtypes = [_vp, _vp, _i64, _i32, _vp, _vp, _vp, _vp]
_lib.msi_knn_dtw.argtypes = [_vp, _vp, _i64, _i32, _i32, _vp, _vp, _vp, _vp]
_lib.msi_index_save.argtypes = [_vp, ctypes.c_char_p]
_lib.msi_index_load.argtypes = [ctypes.c_char_p, _vp, ctypes.POINTER(_BuildOpts), ctypes.POINTER(_vp)]
_lib.msi_knn_ex.restype = ctypes.c_int
_lib.msi_free.argtypes = [_vp]
_lib.msi_free.restype = None
_lib.msi_status_str.argtypes = [ctypes.c_int]
_lib.msi_status_str.restype = ctypes.c_char_p
_lib.msi_last_error.argtypes = []
_lib.msi_last_error.restype = ctypes.c_char_p
_lib.msi_abi_version.argtypes = []
_lib.msi_abi_version.restype = _i32
_lib.msi_index_info_get.argtypes = [_vp, ctypes.POINTER(_IndexInfo)]
_lib.msi_index_info_get.restype = ctypes.c_int
_lib.msi_index_export.argtypes = [_vp, ctypes.POINTER(_Export)]
_lib.msi_index_export.restype = ctypes.c_int
_lib.msi_lower_bounds.argtypes = [_vp, _vp, _vp, _vp, _vp]
_lib.msi_lower_bounds.restype = ctypes.c_int
_lib.msi_query_stats_get.argtypes = [_vp, ctypes.POINTER(_QueryStats), _i32]
_lib.msi_query_stats_get.restype = ctypes.c_int
_lib.msi_set_timing.argtypes = [_vp, _i32]
_lib.msi_set_timing.restype = ctypes.c_int
_lib.msi_lower_bounds_noalloc.argtypes = [_vp, _vp, _vp, _vp, _vp]
_lib.msi_lower_bounds_noalloc.restype = ctypes.c_int
_lib.msi_schedule_set.argtypes = [_vp, _vp]
_lib.msi_schedule_set.restype = ctypes.c_int
_lib.msi_schedule_get.argtypes = [_vp, _vp]
_lib.msi_schedule_get.restype = ctypes.c_int
_lib.msi_merge_topk.argtypes = [_vp, _vp, _i32, _i64, _i32, _i32, _vp, _vp, _vp, _vp]
_lib.msi_merge_topk.restype = ctypes.c_int


class _ServerOpts(ctypes.Structure):
    _fields_ = [("slots_per_index", ctypes.c_int32), ("workspace_bytes", ctypes.c_int64),
                ("max_inflight", ctypes.c_int32), ("slot_capacity", ctypes.c_int32)]


_lib.msi_server_create.argtypes = [_vp, _i32, ctypes.POINTER(_ServerOpts), ctypes.POINTER(_vp)]
_lib.msi_server_create.restype = ctypes.c_int
_lib.msi_server_submit.argtypes = [_vp, _i32, _vp, _i32, ctypes.POINTER(ctypes.c_uint64)]
_lib.msi_server_submit.restype = ctypes.c_int
_lib.msi_server_wait.argtypes = [_vp, ctypes.c_uint64, _vp, _vp, ctypes.POINTER(ctypes.c_double)]
_lib.msi_server_wait.restype = ctypes.c_int
_lib.msi_server_stats.argtypes = [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i32)]
_lib.msi_server_stats.restype = ctypes.c_int
_lib.msi_server_free.argtypes = [_vp]
_lib.msi_server_free.restype = None


class MsiError(RuntimeError):
    def __init__(self, status, detail):
        self.status = status
        super().__init__(f"{msi_status_str(status)}: {detail}")


def _check(status):
    if status != MSI_OK:
        raise MsiError(status, msi_last_error())


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """Raw pointer of a contiguous numpy array or torch tensor of `dtype`."""
    if x is None:
        return None
    if _is_torch(x):
        import torch
        want = {np.float32: torch.float32, np.int64: torch.int64}[dtype]
        if x.dtype != want or not x.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor")
        return ctypes.c_void_p(x.data_ptr())
    if not isinstance(x, np.ndarray) or x.dtype != dtype or not x.flags["C_CONTIGUOUS"]:
        raise TypeError(f"expected a C-contiguous numpy {np.dtype(dtype)} array")
    return ctypes.c_void_p(x.ctypes.data)


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Index:
    """Owner of an msi_index handle; msi_free runs when it is released."""

    def __init__(self, handle, keepalive=None):
        self.handle = handle
        self._keepalive = keepalive  # borrowed collection
        info = msi_index_info_get(self)
        self.n, self.len, self.segments = info["n"], info["len"], info["segments"]
        self.cardinality, self.leaves = info["cardinality"], info["leaves"]

    def close(self):
        if self.handle:
            msi_free(self)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- entry points
def msi_status_str(status):
    return _lib.msi_status_str(int(status)).decode()


def msi_last_error():
    return _lib.msi_last_error().decode()


def msi_abi_version():
    return int(_lib.msi_abi_version())


def msi_build(series, n=None, len=None, segments=16, cardinality=256, leaf_capacity=0, flags=0, stream=None,
              query_slots=0, slot_capacity=0):
    """msi_build: `series` is float32 [n, len] (numpy host array or torch tensor, host
    or device). Returns an Index."""
    n = series.shape[0] if n is None else n
    len_ = series.shape[1] if len is None else len
    opts = _BuildOpts(leaf_capacity, flags, _stream(stream), query_slots, slot_capacity)
    out = ctypes.c_void_p()
    _check(_lib.msi_build(_ptr(series, np.float32), n, len_, segments, cardinality, ctypes.byref(opts),
                          ctypes.byref(out)))
    return Index(out.value, keepalive=series if flags & MSI_BUILD_BORROW else None)


def msi_knn(index, queries, k, ids=None, dists=None, stream=None, nq=None):
    """msi_knn: `queries` float32 [nq, len] host or device. Outputs are allocated
    like the queries (numpy for host input, torch on the same device otherwise)
    unless given. Returns (ids int64 [nq, k], dists float32 [nq, k])."""
    nq = queries.shape[0] if nq is None else nq
    if ids is None:
        if _is_torch(queries):
            import torch
            ids = torch.empty((nq, k), dtype=torch.int64, device=queries.device)
            dists = torch.empty((nq, k), dtype=torch.float32, device=queries.device) if dists is None else dists
        else:
            ids = np.empty((nq, k), dtype=np.int64)
            dists = np.empty((nq, k), dtype=np.float32) if dists is None else dists
    _check(_lib.msi_knn(ctypes.c_void_p(index.handle), _ptr(queries, np.float32), nq, k, _ptr(ids, np.int64),
                        _ptr(dists, np.float32), _stream(stream)))
    return ids, dists


def msi_knn_ex(index, queries, k, stream=None):
    """msi_knn_ex: (ids int64 [nq, k], dists float32 [nq, k], sqdists64 float64 [nq, k]),
    outputs allocated like the queries (numpy for host input, torch on its device)."""
    nq = queries.shape[0]
    if _is_torch(queries):
        import torch
        ids = torch.empty((nq, k), dtype=torch.int64, device=queries.device)
        dists = torch.empty((nq, k), dtype=torch.float32, device=queries.device)
        d64 = torch.empty((nq, k), dtype=torch.float64, device=queries.device)
        d64p = ctypes.c_void_p(d64.data_ptr())
    else:
        ids = np.empty((nq, k), dtype=np.int64)
        dists = np.empty((nq, k), dtype=np.float32)
        d64 = np.empty((nq, k), dtype=np.float64)
        d64p = ctypes.c_void_p(d64.ctypes.data)
    _check(_lib.msi_knn_ex(ctypes.c_void_p(index.handle), _ptr(queries, np.float32), nq, k, _ptr(ids, np.int64),
                           _ptr(dists, np.float32), d64p, _stream(stream)))
    return ids, dists, d64


def msi_index_save(index, path):
    """msi_index_save: writes the index (and an owned collection) to `path`."""
    _check(_lib.msi_index_save(ctypes.c_void_p(index.handle), os.fsencode(path)))


def msi_index_load(path, series=None, query_slots=0, slot_capacity=0, stream=None):
    """msi_index_load: an Index read from `path`; `series` is the same device
    collection for an index saved from a borrowed collection, else None."""
    opts = _BuildOpts(0, 0, _stream(stream), query_slots, slot_capacity)
    out = ctypes.c_void_p()
    _check(_lib.msi_index_load(os.fsencode(path), _ptr(series, np.float32) if series is not None else None,
                               ctypes.byref(opts), ctypes.byref(out)))
    return Index(out.value, keepalive=series)


def msi_knn_dtw(index, queries, k, window=None, stream=None):
    """msi_knn_dtw: exact k-NN under DTW with a Sakoe-Chiba window of half-width
    `window` points (default len // 10). Returns (ids, dists, sqdists64) like msi_knn_ex."""
    if window is None:
        window = index.len // 10
    nq = queries.shape[0]
    if _is_torch(queries):
        import torch
        ids = torch.empty((nq, k), dtype=torch.int64, device=queries.device)
        dists = torch.empty((nq, k), dtype=torch.float32, device=queries.device)
        d64 = torch.empty((nq, k), dtype=torch.float64, device=queries.device)
        d64p = ctypes.c_void_p(d64.data_ptr())
    else:
        ids = np.empty((nq, k), dtype=np.int64)
        dists = np.empty((nq, k), dtype=np.float32)
        d64 = np.empty((nq, k), dtype=np.float64)
        d64p = ctypes.c_void_p(d64.ctypes.data)
    _check(_lib.msi_knn_dtw(ctypes.c_void_p(index.handle), _ptr(queries, np.float32), nq, k, int(window),
                            _ptr(ids, np.int64), _ptr(dists, np.float32), d64p, _stream(stream)))
    return ids, dists, d64


def msi_free(index):
    _lib.msi_free(ctypes.c_void_p(index.handle if isinstance(index, Index) else index))


def msi_index_info_get(index):
    info = _IndexInfo()
    _check(_lib.msi_index_info_get(ctypes.c_void_p(index.handle), ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in _IndexInfo._fields_}


def msi_index_export(index, words=True, perm=True, leaves=True, thresholds=True, znorm=False, fine=False):
    """msi_index_export into fresh numpy arrays (a dict); `fine` gives the fine PAA as
    float16 [n, fine_segments] in collection order (absent when the index keeps none)."""
    n, w, L = index.n, index.segments, index.leaves
    out = {}
    wf = msi_index_info_get(index)["fine_segments"]
    if fine and wf:
        out["fine"] = np.empty((n, wf), dtype=np.float16)
    if words:
        out["words"] = np.empty((n, w), dtype=np.uint8)
    if perm:
        out["perm"] = np.empty(n, dtype=np.uint32)
    if leaves:
        out["leaf_begin"] = np.empty(L + 1, dtype=np.uint32)
        out["env_lo"] = np.empty((L, w), dtype=np.uint8)
        out["env_hi"] = np.empty((L, w), dtype=np.uint8)
    if thresholds:
        out["thresholds"] = np.empty(index.cardinality - 1, dtype=np.float32)
    if znorm:
        out["znorm"] = np.empty((n, index.len), dtype=np.float32)
    ex = _Export(*[ctypes.c_void_p(out[f].ctypes.data) if f in out else None for f, _ in _Export._fields_])
    _check(_lib.msi_index_export(ctypes.c_void_p(index.handle), ctypes.byref(ex)))
    return out


def msi_lower_bounds(index, query, stream=None):
    """msi_lower_bounds: (series_lb float32 [n] in collection order, leaf_lb float32 [leaves])."""
    s = np.empty(index.n, dtype=np.float32)
    lf = np.empty(index.leaves, dtype=np.float32)
    _check(_lib.msi_lower_bounds(ctypes.c_void_p(index.handle), _ptr(query, np.float32), _ptr(s, np.float32),
                                 _ptr(lf, np.float32), _stream(stream)))
    return s, lf


def msi_query_stats_get(index, reset=False):
    st = _QueryStats()
    _check(_lib.msi_query_stats_get(ctypes.c_void_p(index.handle), ctypes.byref(st), 1 if reset else 0))
    return {f: getattr(st, f) for f, _ in _QueryStats._fields_}


def msi_set_timing(index, enable=True):
    _check(_lib.msi_set_timing(ctypes.c_void_p(index.handle), 1 if enable else 0))


class _TuneResult(ctypes.Structure):
    _fields_ = [("query_slots", ctypes.c_int32), ("grid_share", ctypes.c_int32), ("queries_per_s", ctypes.c_double),
                ("candidates", ctypes.c_int32), ("default_queries_per_s", ctypes.c_double),
                ("batch_chain", ctypes.c_int32), ("batch_group", ctypes.c_int32), ("batch_share", ctypes.c_int32),
                ("batch_dense", ctypes.c_int32)]


class _Schedule(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int32) for f in ("batch_chain", "query_slots", "grid_share", "batch_group",
                                              "batch_share", "batch_overlap", "batch_dense", "batch_order")]


def msi_autotune(index, queries, k, reps=0, stream=None):
    """msi_autotune: times the batched schedules (batched chain and query slots) on
    `queries` [nq >= 2, len] (host or device) and keeps the fastest for the index.
    Returns the choice as a dict."""
    out = _TuneResult()
    _check(_lib.msi_autotune(ctypes.c_void_p(index.handle), _ptr(queries, np.float32), queries.shape[0], k, reps,
                             ctypes.byref(out), _stream(stream)))
    return {f: getattr(out, f) for f, _ in _TuneResult._fields_}


def msi_schedule_get(index):
    """msi_schedule_get: the index's batched schedule as a dict."""
    sc = _Schedule()
    _check(_lib.msi_schedule_get(ctypes.c_void_p(index.handle), ctypes.byref(sc)))
    return {f: getattr(sc, f) for f, _ in _Schedule._fields_}


def msi_schedule_set(index, **changes):
    """msi_schedule_set: changes the named fields of the index's batched schedule
    (batch_chain, query_slots, grid_share, batch_group, batch_share, batch_overlap,
    batch_dense, batch_order)."""
    cur = msi_schedule_get(index)
    unknown = set(changes) - set(cur)
    if unknown:
        raise TypeError(f"unknown schedule fields {sorted(unknown)}")
    cur.update(changes)
    sc = _Schedule(**{f: int(v) for f, v in cur.items()})
    _check(_lib.msi_schedule_set(ctypes.c_void_p(index.handle), ctypes.byref(sc)))


def msi_lower_bounds_noalloc(index, query, series_lb, leaf_lb, stream=None):
    """msi_lower_bounds_noalloc: device tensors only (query float32 [len], outputs
    float32 [n] and [leaves]); the library allocates nothing for this call."""
    _check(_lib.msi_lower_bounds_noalloc(ctypes.c_void_p(index.handle), _ptr(query, np.float32),
                                         _ptr(series_lb, np.float32), _ptr(leaf_lb, np.float32), _stream(stream)))


def msi_merge_topk(ids, sqdists64, k, stream=None):
    """msi_merge_topk: ids int64 [parts, nq, k_in] and sqdists64 float64 [parts, nq,
    k_in] (each row sorted by (distance, id), ids distinct across parts), numpy or
    torch. Returns (ids int64 [nq, k], dists float32 [nq, k], sqdists64 [nq, k]),
    allocated like `ids` (numpy, or torch on its device)."""
    parts, nq, kin = ids.shape
    if _is_torch(ids):
        import torch
        if sqdists64.dtype != torch.float64 or not sqdists64.is_contiguous():
            raise TypeError("expected a contiguous float64 tensor of distances")
        oi = torch.empty((nq, k), dtype=torch.int64, device=ids.device)
        od = torch.empty((nq, k), dtype=torch.float32, device=ids.device)
        o64 = torch.empty((nq, k), dtype=torch.float64, device=ids.device)
        dp, o64p = ctypes.c_void_p(sqdists64.data_ptr()), ctypes.c_void_p(o64.data_ptr())
    else:
        sqdists64 = np.ascontiguousarray(sqdists64, dtype=np.float64)
        oi = np.empty((nq, k), dtype=np.int64)
        od = np.empty((nq, k), dtype=np.float32)
        o64 = np.empty((nq, k), dtype=np.float64)
        dp, o64p = ctypes.c_void_p(sqdists64.ctypes.data), ctypes.c_void_p(o64.ctypes.data)
    _check(_lib.msi_merge_topk(_ptr(ids, np.int64), dp, parts, nq, kin, k, _ptr(oi, np.int64), _ptr(od, np.float32),
                               o64p, _stream(stream)))
    return oi, od, o64


class Server:
    """msi_server_*: a request loop with continuous batching over resident indexes."""

    def __init__(self, indexes, slots_per_index=0, workspace_bytes=0, max_inflight=0, slot_capacity=0):
        self._indexes = list(indexes)  # keep the indexes alive
        arr = (ctypes.c_void_p * len(self._indexes))(*[ix.handle for ix in self._indexes])
        opts = _ServerOpts(slots_per_index, workspace_bytes, max_inflight, slot_capacity)
        out = ctypes.c_void_p()
        _check(_lib.msi_server_create(ctypes.cast(arr, ctypes.c_void_p), len(self._indexes), ctypes.byref(opts),
                                      ctypes.byref(out)))
        self.handle = out.value

    def submit(self, index_no, query, k):
        """msi_server_submit: query is a host float32 array of the index's length."""
        q = np.ascontiguousarray(query, dtype=np.float32)
        t = ctypes.c_uint64()
        _check(_lib.msi_server_submit(ctypes.c_void_p(self.handle), index_no, ctypes.c_void_p(q.ctypes.data), k,
                                      ctypes.byref(t)))
        return t.value

    def wait(self, ticket, k):
        """msi_server_wait: (ids int64 [k], dists float32 [k], latency ms)."""
        ids = np.empty(k, dtype=np.int64)
        d = np.empty(k, dtype=np.float32)
        ms = ctypes.c_double()
        _check(_lib.msi_server_wait(ctypes.c_void_p(self.handle), ticket, ctypes.c_void_p(ids.ctypes.data),
                                    ctypes.c_void_p(d.ctypes.data), ctypes.byref(ms)))
        return ids, d, ms.value

    def stats(self):
        c, r, sl = _i64(), _i64(), _i32()
        _check(_lib.msi_server_stats(ctypes.c_void_p(self.handle), ctypes.byref(c), ctypes.byref(r), ctypes.byref(sl)))
        return {"completed": c.value, "reruns": r.value, "slots": sl.value}

    def close(self):
        if self.handle:
            _lib.msi_server_free(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
