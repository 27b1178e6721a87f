"""ctypes binding of librmq_gb300.so (include/rmq.h), argument marshalling only.

Functions carry the C ABI's names.  Device arrays are torch CUDA tensors
(their data pointers are passed through); host arrays are numpy arrays; the
stream defaults to torch's current stream on the tensor's device.  Every
step of the computation runs in the library's CUDA kernels; if the library
is missing this module raises instead of computing anything itself.

Calls that return an rmq_status raise RmqError for anything but RMQ_OK,
except rmq_stream_status, which returns the status.
"""
from __future__ import annotations

import ctypes
import enum
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librmq_gb300.so")


class Status(enum.IntEnum):
    OK = 0
    ERR_INVALID_ARG = 1
    ERR_QUERY_RANGE = 2
    ERR_OOM = 3
    ERR_CUDA = 4
    ERR_TIMEOUT = 5
    ERR_BUDGET = 6
    ERR_SCRATCH_LIMIT = 7


class Variant(enum.IntEnum):
    AUTO = 0
    PLAIN = 1
    CONTRACTED = 2


class RmqError(RuntimeError):
    def __init__(self, status):
        self.status = Status(status)
        super().__init__("%s: %s" % (self.status.name, strerror(self.status)))


FLAG_TEST_WITHHOLD_READY = 1


class rmq_array(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("n", ctypes.c_int64), ("q", ctypes.c_int64)]


class rmq_server_opts(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("inflight", ctypes.c_int32),
                ("max_batch_queries", ctypes.c_int32), ("flags", ctypes.c_int32), ("pad", ctypes.c_int32)]


class rmq_server_stats(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_int64), ("queries", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("table_bytes_in_use", ctypes.c_int64), ("resident_arrays", ctypes.c_int64)]


class rmq_scan_stats(ctypes.Structure):
    _fields_ = [("open_queries", ctypes.c_int64), ("table_reads", ctypes.c_int64), ("m1_reads", ctypes.c_int64),
                ("scan_elems", ctypes.c_int64), ("rank_reads", ctypes.c_int64)]


class rmq_opts(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("k", ctypes.c_int32),
                ("k_con", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("threads_per_query", ctypes.c_int32), ("k1", ctypes.c_int32)]


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_SIGS = {
    "rmq_batch": (_i32, [_vp, _i64, _vp, _vp, _i64, _vp, _vp]),
    "rmq_batch_ex": (_i32, [_vp, _i64, _vp, _vp, _i64, _vp, ctypes.POINTER(rmq_opts), _vp]),
    "rmq_batch_timed": (_i32, [_vp, _i64, _vp, _vp, _i64, _vp, ctypes.POINTER(rmq_opts), _vp,
                               ctypes.POINTER(_vp), _i32]),
    "rmq_launch_count": (_i64, []),
    "rmq_batch_counted": (_i32, [_vp, _i64, _vp, _vp, _i64, _vp, ctypes.POINTER(rmq_opts), _vp,
                                 ctypes.POINTER(rmq_scan_stats)]),
    "rmq_batch_noalloc": (_i32, [_vp, _i64, _vp, _vp, _i64, _vp, _i32, _vp]),
    "rmq_batch_multi": (_i32, [ctypes.c_void_p, _i32, _vp, _vp, _vp, ctypes.POINTER(rmq_opts), _vp]),
    "rmq_autotune": (_i32, [_vp, _i64, _vp, _vp, _i64, _vp, _i32, _i32, _i32, _vp, ctypes.POINTER(rmq_opts),
                            ctypes.POINTER(ctypes.c_float)]),
    "rmq_tune_save": (_i32, [ctypes.c_char_p]),
    "rmq_tune_load": (_i32, [ctypes.c_char_p]),
    "rmq_tune_clear": (None, []),
    "rmq_query_multi": (_i32, [_vp, _vp, _i32, _vp, _vp, _vp, _vp]),
    "rmq_server_create": (_i32, [ctypes.POINTER(rmq_server_opts), ctypes.POINTER(_vp)]),
    "rmq_server_admit": (_i32, [_vp, _vp, _i64, _i32, ctypes.POINTER(_i32)]),
    "rmq_server_admit_wait": (_i32, [_vp, _vp, _i64, _i32, ctypes.c_double, ctypes.POINTER(_i32)]),
    "rmq_server_evict": (_i32, [_vp, _i32]),
    "rmq_server_submit": (_i32, [_vp, _i32, _vp, _vp, _i64, _vp, ctypes.POINTER(_i64)]),
    "rmq_server_wait": (_i32, [_vp, _i64, ctypes.POINTER(ctypes.c_double)]),
    "rmq_server_stats_get": (_i32, [_vp, ctypes.POINTER(rmq_server_stats)]),
    "rmq_server_destroy": (None, [_vp]),
    "rmq_batch_host": (_i32, [_vp, _i64, _vp, _vp, _i64, _vp, ctypes.POINTER(rmq_opts), _vp]),
    "rmq_build": (_i32, [_vp, _i64, ctypes.POINTER(rmq_opts), _vp, ctypes.POINTER(_vp)]),
    "rmq_query": (_i32, [_vp, _vp, _vp, _i64, _vp, _vp]),
    "rmq_query_host": (_i32, [_vp, _vp, _vp, _i64, _vp, _vp]),
    "rmq_handle_bytes": (_i64, [_vp]),
    "rmq_handle_k": (_i32, [_vp]),
    "rmq_free": (None, [_vp]),
    "rmq_stream_status": (_i32, [_vp]),
    "rmq_strerror": (ctypes.c_char_p, [_i32]),
    "rmq_table_bytes": (_i64, [_i64, _i32]),
    "rmq_batch_workspace_bytes": (_i64, [_i64, _i64, ctypes.POINTER(rmq_opts)]),
    "rmq_batch_lary": (_i32, [_vp, _i64, _vp, _vp, _i64, _vp, _i32, _i32, _vp]),
    "rmq_batch_hlevel": (_i32, [_vp, _i64, _vp, _vp, _i64, _vp, _vp, _i32, _vp]),
    "rmq_hlevel_bytes": (_i64, [_i64, _vp, _i32]),
    "rmq_hlevel_paper_ks": (_i32, [_i64, _i32, _vp]),
    "rmq_tune": (_i32, [_i64, _i64, ctypes.POINTER(rmq_opts)]),
    "rmq_tune_batch": (_i32, [_vp, _vp, _i64, _i64, _vp, ctypes.POINTER(rmq_opts)]),
    "rmq_block_minima": (_i32, [_vp, _i64, _i32, _vp, _vp]),
    "rmq_sparse_table_build": (_i32, [_vp, _i64, _vp]),
    "rmq_sort_endpoints": (_i32, [_vp, _vp, _i64, _i64, _vp, _vp, _vp]),
    "rmq_rank_endpoints": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp]),
    "rmq_contract": (_i32, [_vp, _i64, _vp, _vp, _i64, _vp, _vp]),
    "rmq_endpoint_bitmap": (_i32, [_vp, _vp, _i64, _i64, _vp, _vp, _vp]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("librmq_gb300.so not found at %s: run __graft_entry__.build() "
                           "(the library has no CPU fallback)" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


def strerror(status) -> str:
    return load().rmq_strerror(int(status)).decode()


def _check(st):
    if st != 0:
        raise RmqError(st)


def _opts(variant=0, k=0, k_con=0, flags=0, threads_per_query=0, k1=0):
    return rmq_opts(int(variant), int(k), int(k_con), int(flags), int(threads_per_query), int(k1))


def _opts_dict(o) -> dict:
    return {"variant": Variant(o.variant), "k": o.k, "k_con": o.k_con,
            "threads_per_query": o.threads_per_query, "k1": o.k1}


def _stream(stream, t=None):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    dev = t.device if t is not None else None
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _dptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise ValueError("%s must have dtype %s" % (name, dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr()) if t.numel() else ctypes.c_void_p(0)


def _i32t():
    import torch
    return torch.int32


# ---------------------------------------------------------------- batch

def rmq_batch(A, l, r, out, stream=None):
    """out[i] = leftmost argmin of A[l[i]..r[i]] (tuned form and k)."""
    _check(load().rmq_batch(_dptr(A, _i32t(), "A"), A.numel(), _dptr(l, _i32t(), "l"),
                            _dptr(r, _i32t(), "r"), l.numel(), _dptr(out, _i32t(), "out"),
                            _stream(stream, A)))


def rmq_batch_ex(A, l, r, out, variant=0, k=0, k_con=0, stream=None, flags=0, threads_per_query=0, k1=0):
    o = _opts(variant, k, k_con, flags, threads_per_query, k1)
    _check(load().rmq_batch_ex(_dptr(A, _i32t(), "A"), A.numel(), _dptr(l, _i32t(), "l"),
                               _dptr(r, _i32t(), "r"), l.numel(), _dptr(out, _i32t(), "out"),
                               ctypes.byref(o), _stream(stream, A)))


def rmq_batch_timed(A, l, r, out, events, variant=0, k=0, k_con=0, stream=None, threads_per_query=0, k1=0):
    """rmq_batch_ex recording torch.cuda.Event objects at the stage boundaries
    (4 for the plain form, 6 for the contracted form, whose optional 7th is
    recorded after the bitmap clear inside step 1)."""
    handles = []
    for ev in events:
        if ev.cuda_event == 0:       # torch creates the CUDA event lazily
            ev.record()
        handles.append(ev.cuda_event)
    arr = (ctypes.c_void_p * max(len(handles), 1))(*handles)
    o = _opts(variant, k, k_con, 0, threads_per_query, k1)
    _check(load().rmq_batch_timed(_dptr(A, _i32t(), "A"), A.numel(), _dptr(l, _i32t(), "l"),
                                  _dptr(r, _i32t(), "r"), l.numel(), _dptr(out, _i32t(), "out"),
                                  ctypes.byref(o), _stream(stream, A), arr, len(handles)))


def rmq_batch_counted(A, l, r, out, variant=0, k=0, k_con=0, stream=None, threads_per_query=0, k1=0) -> dict:
    """rmq_batch_ex through the instrumented query kernel; returns the work
    counts of the open queries (rmq_scan_stats as a dict).  Waits."""
    o = _opts(variant, k, k_con, 0, threads_per_query, k1)
    st = rmq_scan_stats()
    _check(load().rmq_batch_counted(_dptr(A, _i32t(), "A"), A.numel(), _dptr(l, _i32t(), "l"),
                                    _dptr(r, _i32t(), "r"), l.numel(), _dptr(out, _i32t(), "out"),
                                    ctypes.byref(o), _stream(stream, A), ctypes.byref(st)))
    return {f: int(getattr(st, f)) for f, _ in rmq_scan_stats._fields_}


def rmq_batch_noalloc(A, l, r, out, k=0, stream=None):
    """Plain-form batch whose table sits in the library's fixed device buffer
    (no device allocation); see include/rmq.h."""
    _check(load().rmq_batch_noalloc(_dptr(A, _i32t(), "A"), A.numel(), _dptr(l, _i32t(), "l"),
                                    _dptr(r, _i32t(), "r"), l.numel(), _dptr(out, _i32t(), "out"),
                                    int(k), _stream(stream, A)))


def rmq_batch_multi(arrays, qs, l, r, out, k=0, flags=0, stream=None):
    """Many arrays in one launch.  arrays: list of int32 CUDA tensors; qs: number
    of queries of each (consecutive in l, r, out; positions relative to the array)."""
    H = len(arrays)
    desc = (rmq_array * max(H, 1))()
    for h, (A, q) in enumerate(zip(arrays, qs)):
        desc[h] = rmq_array(ctypes.c_void_p(_dptr(A, _i32t(), "A").value), A.numel(), int(q))
    o = _opts(0, k, 0, flags)
    dev = arrays[0] if H else l
    _check(load().rmq_batch_multi(ctypes.cast(desc, ctypes.c_void_p), H, _dptr(l, _i32t(), "l"),
                                  _dptr(r, _i32t(), "r"), _dptr(out, _i32t(), "out"), ctypes.byref(o),
                                  _stream(stream, dev)))


def rmq_launch_count() -> int:
    return int(load().rmq_launch_count())


def rmq_batch_host(A, l, r, out, variant=0, k=0, k_con=0, stream=None, threads_per_query=0, k1=0):
    """Host-buffer batch (numpy int32 arrays, out written in place); waits."""
    for name, a in (("A", A), ("l", l), ("r", r), ("out", out)):
        if not (isinstance(a, np.ndarray) and a.dtype == np.int32 and a.flags.c_contiguous):
            raise ValueError("%s must be a C-contiguous numpy int32 array" % name)
    o = _opts(variant, k, k_con, 0, threads_per_query, k1)
    st = load().rmq_batch_host(A.ctypes.data, len(A), l.ctypes.data, r.ctypes.data, len(l),
                               out.ctypes.data, ctypes.byref(o), _stream(stream))
    _check(st)


# ---------------------------------------------------------------- handles

class Handle:
    """A resident plain-BbST structure (rmq_build).  A is borrowed: the
    tensor is kept referenced here so it outlives the handle."""

    def __init__(self, ptr, A):
        self.ptr = ptr
        self.A = A

    @property
    def bytes(self) -> int:
        return int(load().rmq_handle_bytes(self.ptr))

    @property
    def k(self) -> int:
        return int(load().rmq_handle_k(self.ptr))

    def free(self):
        if self.ptr:
            load().rmq_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def rmq_build(A, k=0, stream=None) -> Handle:
    h = ctypes.c_void_p()
    o = _opts(0, k, 0)
    _check(load().rmq_build(_dptr(A, _i32t(), "A"), A.numel(), ctypes.byref(o),
                            _stream(stream, A), ctypes.byref(h)))
    return Handle(h, A)


def rmq_query(h: Handle, l, r, out, stream=None):
    _check(load().rmq_query(h.ptr, _dptr(l, _i32t(), "l"), _dptr(r, _i32t(), "r"), l.numel(),
                            _dptr(out, _i32t(), "out"), _stream(stream, l)))


def rmq_query_host(h: Handle, l, r, out, stream=None):
    """One request on host buffers (numpy int32; out written in place); waits."""
    for name, a in (("l", l), ("r", r), ("out", out)):
        if not (isinstance(a, np.ndarray) and a.dtype == np.int32 and a.flags.c_contiguous):
            raise ValueError("%s must be a C-contiguous numpy int32 array" % name)
    _check(load().rmq_query_host(h.ptr, l.ctypes.data, r.ctypes.data, len(l), out.ctypes.data, _stream(stream)))


def rmq_query_multi(handles, qs, l, r, out, stream=None):
    """Queries of several requests against resident handles in one launch."""
    H = len(handles)
    hs = (ctypes.c_void_p * max(H, 1))(*[h.ptr.value if isinstance(h.ptr, ctypes.c_void_p) else h.ptr
                                         for h in handles])
    qc = (ctypes.c_int64 * max(H, 1))(*[int(q) for q in qs])
    _check(load().rmq_query_multi(ctypes.cast(hs, ctypes.c_void_p), ctypes.cast(qc, ctypes.c_void_p), H,
                                  _dptr(l, _i32t(), "l"), _dptr(r, _i32t(), "r"), _dptr(out, _i32t(), "out"),
                                  _stream(stream, l)))


class Server:
    """The library's continuous-batching server (rmq_server_*).  Requests use
    host numpy int32 arrays, kept referenced here until their ticket is waited."""

    def __init__(self, budget_bytes=0, inflight=0, max_batch_queries=0):
        o = rmq_server_opts(int(budget_bytes), int(inflight), int(max_batch_queries), 0, 0)
        self.ptr = ctypes.c_void_p()
        _check(load().rmq_server_create(ctypes.byref(o), ctypes.byref(self.ptr)))
        self._arrays = {}
        self._live = {}

    def admit(self, A, k=0) -> int:
        i = ctypes.c_int32()
        _check(load().rmq_server_admit(self.ptr, _dptr(A, _i32t(), "A"), A.numel(), int(k), ctypes.byref(i)))
        self._arrays[i.value] = A
        return i.value

    def admit_wait(self, A, timeout_s, k=0) -> int:
        """admit, waiting up to timeout_s seconds for evictions to free budget."""
        i = ctypes.c_int32()
        _check(load().rmq_server_admit_wait(self.ptr, _dptr(A, _i32t(), "A"), A.numel(), int(k),
                                            float(timeout_s), ctypes.byref(i)))
        self._arrays[i.value] = A
        return i.value

    def evict(self, array_id):
        _check(load().rmq_server_evict(self.ptr, int(array_id)))
        self._arrays.pop(array_id, None)

    def submit(self, array_id, l, r, out) -> int:
        for name, a in (("l", l), ("r", r), ("out", out)):
            if not (isinstance(a, np.ndarray) and a.dtype == np.int32 and a.flags.c_contiguous):
                raise ValueError("%s must be a C-contiguous numpy int32 array" % name)
        t = ctypes.c_int64()
        _check(load().rmq_server_submit(self.ptr, int(array_id), l.ctypes.data, r.ctypes.data, len(l),
                                        out.ctypes.data, ctypes.byref(t)))
        self._live[t.value] = (l, r, out)
        return t.value

    def wait(self, ticket) -> float:
        lat = ctypes.c_double()
        st = load().rmq_server_wait(self.ptr, int(ticket), ctypes.byref(lat))
        self._live.pop(ticket, None)
        _check(st)
        return lat.value

    def stats(self) -> dict:
        s = rmq_server_stats()
        _check(load().rmq_server_stats_get(self.ptr, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in rmq_server_stats._fields_}

    def close(self):
        if self.ptr:
            load().rmq_server_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rmq_free(h: Handle):
    h.free()


def rmq_handle_bytes(h: Handle) -> int:
    return h.bytes


# ---------------------------------------------------------------- diagnostics

def rmq_stream_status(stream=None) -> Status:
    return Status(load().rmq_stream_status(_stream(stream)))


def rmq_strerror(status) -> str:
    return strerror(status)


def rmq_table_bytes(n: int, k: int) -> int:
    return int(load().rmq_table_bytes(int(n), int(k)))


def rmq_batch_lary(A, l, r, out, k: int, ell: int, stream=None):
    """The plain form over the ell-ary block sparse table (see include/rmq.h)."""
    _check(load().rmq_batch_lary(_dptr(A, _i32t(), "A"), A.numel(), _dptr(l, _i32t(), "l"),
                                 _dptr(r, _i32t(), "r"), l.numel(), _dptr(out, _i32t(), "out"),
                                 int(k), int(ell), _stream(stream, A)))


def _ks_array(ks):
    ks = [int(k) for k in ks]
    return (ctypes.c_int32 * max(1, len(ks)))(*ks), len(ks)


def rmq_batch_hlevel(A, l, r, out, ks, stream=None):
    """The plain form over the multi-level block sparse table of Sec. 3.3,
    block sizes ks = (k_1, ..., k_h) (see include/rmq.h)."""
    arr, h = _ks_array(ks)
    _check(load().rmq_batch_hlevel(_dptr(A, _i32t(), "A"), A.numel(), _dptr(l, _i32t(), "l"),
                                   _dptr(r, _i32t(), "r"), l.numel(), _dptr(out, _i32t(), "out"),
                                   ctypes.cast(arr, ctypes.c_void_p), h, _stream(stream, A)))


def rmq_hlevel_bytes(n: int, ks) -> int:
    """Bytes of the multi-level structure for n and ks (-1 on bad arguments)."""
    arr, h = _ks_array(ks)
    return int(load().rmq_hlevel_bytes(int(n), ctypes.cast(arr, ctypes.c_void_p), h))


def rmq_hlevel_paper_ks(n: int, h: int) -> tuple:
    """Sec. 3.3's block sizes for n and h, rounded to powers of two."""
    arr = (ctypes.c_int32 * max(1, int(h)))()
    _check(load().rmq_hlevel_paper_ks(int(n), int(h), ctypes.cast(arr, ctypes.c_void_p)))
    return tuple(int(x) for x in arr[:int(h)])


def rmq_batch_workspace_bytes(n: int, q: int, variant=0, k=0, k_con=0, threads_per_query=0, k1=0) -> int:
    """Device workspace of one rmq_batch_ex call (-1 on bad arguments)."""
    o = _opts(variant, k, k_con, 0, threads_per_query, k1)
    return int(load().rmq_batch_workspace_bytes(int(n), int(q), ctypes.byref(o)))


def rmq_tune(n: int, q: int) -> dict:
    o = rmq_opts()
    _check(load().rmq_tune(int(n), int(q), ctypes.byref(o)))
    return _opts_dict(o)


def rmq_tune_batch(l, r, n: int, stream=None) -> dict:
    """The options an AUTO call uses for this batch (may read 256 of its queries back)."""
    o = rmq_opts()
    _check(load().rmq_tune_batch(_dptr(l, _i32t(), "l"), _dptr(r, _i32t(), "r"), l.numel(), int(n),
                                 _stream(stream, l), ctypes.byref(o)))
    return _opts_dict(o)


def rmq_autotune(A, l, r, out, variant=0, k_min=0, k_max=0, stream=None):
    """Measure block sizes / forms on this batch; returns (options dict, ms)."""
    o = rmq_opts()
    ms = ctypes.c_float()
    _check(load().rmq_autotune(_dptr(A, _i32t(), "A"), A.numel(), _dptr(l, _i32t(), "l"), _dptr(r, _i32t(), "r"),
                               l.numel(), _dptr(out, _i32t(), "out"), int(variant), int(k_min), int(k_max),
                               _stream(stream, A), ctypes.byref(o), ctypes.byref(ms)))
    return _opts_dict(o), ms.value


def rmq_tune_save(path):
    _check(load().rmq_tune_save(str(path).encode()))


def rmq_tune_load(path):
    _check(load().rmq_tune_load(str(path).encode()))


def rmq_tune_clear():
    load().rmq_tune_clear()


# ---------------------------------------------------------------- steps

def rmq_block_minima(A, k, T0, stream=None):
    _check(load().rmq_block_minima(_dptr(A, _i32t(), "A"), A.numel(), int(k), _dptr(T0, None, "T0"),
                                   _stream(stream, A)))


def rmq_sparse_table_build(T, nb, stream=None):
    _check(load().rmq_sparse_table_build(_dptr(T, None, "T"), int(nb), _stream(stream, T)))


def rmq_sort_endpoints(l, r, n, pos_out, tag_out, stream=None):
    _check(load().rmq_sort_endpoints(_dptr(l, _i32t(), "l"), _dptr(r, _i32t(), "r"), l.numel(), int(n),
                                     _dptr(pos_out, None, "pos_out"), _dptr(tag_out, None, "tag_out"),
                                     _stream(stream, l)))


def rmq_rank_endpoints(pos_sorted, tag_sorted, q, P_out, m_dev, rank_l, rank_r, stream=None):
    _check(load().rmq_rank_endpoints(_dptr(pos_sorted), _dptr(tag_sorted), int(q), _dptr(P_out),
                                     _dptr(m_dev), _dptr(rank_l), _dptr(rank_r), _stream(stream, pos_sorted)))


def rmq_endpoint_bitmap(l, r, n, BP, m_dev, stream=None):
    """BP: int32/uint32 tensor of 2W words, W = ceil(n / 32) + 1 (the W bit
    words, then the W counts of set bits before each word); m_dev: one int64
    on the device."""
    _check(load().rmq_endpoint_bitmap(_dptr(l, _i32t(), "l"), _dptr(r, _i32t(), "r"), l.numel(), int(n),
                                      _dptr(BP, None, "BP"), _dptr(m_dev, None, "m_dev"), _stream(stream, l)))


def rmq_contract(A, P, m_dev, m_max, AQ, stream=None):
    _check(load().rmq_contract(_dptr(A, _i32t(), "A"), A.numel(), _dptr(P), _dptr(m_dev), int(m_max),
                               _dptr(AQ), _stream(stream, A)))
