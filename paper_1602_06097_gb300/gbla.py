"""Thin ctypes binding over the C ABI in ``include/gbla.h``.

Argument marshalling only: every step of the reduction runs in the CUDA
library ``libgbla.so``.  The library is loaded on first use and there is no
fallback: if it is missing or fails to load, the call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbla.so")

GBLA_OK = 0
GEMM_AUTO, GEMM_TCGEN05, GEMM_SIMT, GEMM_FP64, GEMM_U8 = 0, 1, 2, 3, 4
PATH_AUTO, PATH_DENSE, PATH_SPARSE = 0, 1, 2
ORDER_NEW, ORDER_TRSM_FIRST = 0, 1
ECHELON_AUTO, ECHELON_PANELS, ECHELON_SGE = 0, 1, 2

EXPORTS = ["gbla_reduce", "gbla_reduce_ex", "gbla_free", "gbla_strerror", "gbla_version",
           "gbla_modmatmul", "gbla_pivots", "gbla_multiline", "gbla_pivots_noalloc",
           "gbla_selftest_wait_timeout", "gbla_reduce_batch", "gbla_server_create", "gbla_server_submit",
           "gbla_server_wait", "gbla_server_wait_ex", "gbla_server_poll", "gbla_server_cancel", "gbla_server_get_stats", "gbla_server_destroy",
           "gbla_decode_format2", "gbla_decode_format2_ex", "gbla_spmm", "gbla_pipe_peak",
           "gbla_selftest_fail_alloc_after", "gbla_device_bytes_in_use", "gbla_modmatmul32"]


class CsrIn(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class CsrOut(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("on_device", ctypes.c_int)]


class Options(ctypes.Structure):
    _fields_ = [("want_reduced", ctypes.c_int), ("gemm_variant", ctypes.c_int),
                ("device_ptrs", ctypes.c_int), ("panel_width", ctypes.c_int),
                ("path", ctypes.c_int), ("leaf_width", ctypes.c_int), ("kernel_times", ctypes.c_int),
                ("fl_order", ctypes.c_int), ("autotune", ctypes.c_int), ("echelon", ctypes.c_int)]


def _options(want_reduced, variant, device_ptrs, path=PATH_AUTO, leaf=0, kernel_times=False, order=0,
             autotune=False, echelon=0):
    return Options(1 if want_reduced else 0, int(variant), int(device_ptrs), 0, int(path), int(leaf),
                   1 if kernel_times else 0, int(order), 1 if autotune else 0, int(echelon))


class Stats(ctypes.Structure):
    _fields_ = [("npiv", ctypes.c_int64), ("m_cd", ctypes.c_int64), ("n_d", ctypes.c_int64),
                ("rank_d", ctypes.c_int64), ("ms_split", ctypes.c_double), ("ms_trsm", ctypes.c_double),
                ("ms_schur", ctypes.c_double), ("ms_echelon", ctypes.c_double),
                ("ms_backsub", ctypes.c_double), ("ms_output", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("mod_ops", ctypes.c_double), ("launches", ctypes.c_int64),
                ("schur_mod_ops", ctypes.c_double), ("ms_echelon_back", ctypes.c_double),
                ("path", ctypes.c_int64), ("list_a", ctypes.c_int64), ("list_b", ctypes.c_int64),
                ("leaf_width", ctypes.c_int64), ("schur_exec_mod_ops", ctypes.c_double),
                ("tc_launches", ctypes.c_int64), ("gather_launches", ctypes.c_int64),
                ("tc_ms", ctypes.c_double), ("gather_ms", ctypes.c_double), ("tc_mod_ops", ctypes.c_double),
                ("tc_pair_launches", ctypes.c_int64), ("gather_group_m", ctypes.c_int64),
                ("tune_state", ctypes.c_int64), ("echelon_method", ctypes.c_int64),
                ("d_density", ctypes.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("cancelled", ctypes.c_int64), ("queued", ctypes.c_int64), ("running", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("mem_budget", ctypes.c_size_t), ("mem_in_use", ctypes.c_size_t), ("peak_running", ctypes.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class RequestInfo(ctypes.Structure):
    _fields_ = [("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("device_start_ms", ctypes.c_double), ("device_end_ms", ctypes.c_double),
                ("running_at_start", ctypes.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_CANCELLED = 0, 1, 2, 3


GBLA_E_TIMEOUT, GBLA_E_CANCELLED = 4, 7


class GblaError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} (code {code})")


_lib = None
_lock = threading.Lock()


def load():
    """Open libgbla.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgbla.so not built ({LIB_PATH}); run __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i64, u32, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int
        lib.gbla_reduce.argtypes = [ctypes.POINTER(CsrIn), u32, i32, ctypes.POINTER(CsrOut), ctypes.POINTER(i64)]
        lib.gbla_reduce.restype = i32
        lib.gbla_reduce_ex.argtypes = [ctypes.POINTER(CsrIn), u32, ctypes.POINTER(Options), vp,
                                       ctypes.POINTER(CsrOut), ctypes.POINTER(i64), ctypes.POINTER(Stats)]
        lib.gbla_reduce_ex.restype = i32
        lib.gbla_free.argtypes = [ctypes.POINTER(CsrOut)]
        lib.gbla_free.restype = None
        lib.gbla_strerror.argtypes = [i32]
        lib.gbla_strerror.restype = ctypes.c_char_p
        lib.gbla_version.argtypes = []
        lib.gbla_version.restype = i32
        lib.gbla_modmatmul.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64, u32, i32, i32, vp]
        lib.gbla_modmatmul.restype = i32
        lib.gbla_modmatmul32.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64, u32, i32, vp]
        lib.gbla_modmatmul32.restype = i32
        lib.gbla_pivots.argtypes = [ctypes.POINTER(CsrIn), u32, vp, ctypes.POINTER(i64), vp]
        lib.gbla_spmm.restype = i32
        lib.gbla_selftest_fail_alloc_after.argtypes = [i64]
        lib.gbla_selftest_fail_alloc_after.restype = i32
        lib.gbla_device_bytes_in_use.argtypes = [ctypes.POINTER(i64)]
        lib.gbla_device_bytes_in_use.restype = i32
        lib.gbla_pipe_peak.argtypes = [i32, ctypes.POINTER(ctypes.c_double), vp]
        lib.gbla_pipe_peak.restype = i32
        lib.gbla_spmm.argtypes = [i64, i64, i64, vp, i64, ctypes.POINTER(CsrIn), vp, vp, i64, u32, i32, vp]
        lib.gbla_pivots.restype = i32
        lib.gbla_multiline.argtypes = [ctypes.POINTER(CsrIn), vp, vp, vp, vp]
        lib.gbla_multiline.restype = i32
        lib.gbla_pivots_noalloc.argtypes = [ctypes.POINTER(CsrIn), u32, vp, ctypes.POINTER(i64), vp]
        lib.gbla_pivots_noalloc.restype = i32
        lib.gbla_selftest_wait_timeout.argtypes = [vp]
        lib.gbla_selftest_wait_timeout.restype = i32
        lib.gbla_reduce_batch.argtypes = [i32, ctypes.POINTER(CsrIn), ctypes.POINTER(u32), ctypes.POINTER(Options),
                                          i32, ctypes.POINTER(CsrOut), ctypes.POINTER(i64), ctypes.POINTER(i32)]
        lib.gbla_reduce_batch.restype = i32
        lib.gbla_server_create.argtypes = [ctypes.c_size_t, i32, ctypes.POINTER(vp)]
        lib.gbla_server_create.restype = i32
        lib.gbla_server_submit.argtypes = [vp, ctypes.POINTER(CsrIn), u32, ctypes.POINTER(Options),
                                           ctypes.POINTER(i64)]
        lib.gbla_server_submit.restype = i32
        lib.gbla_server_wait.argtypes = [vp, i64, ctypes.c_double, ctypes.POINTER(CsrOut), ctypes.POINTER(i64),
                                         ctypes.POINTER(ctypes.c_double)]
        lib.gbla_server_wait.restype = i32
        lib.gbla_server_wait_ex.argtypes = [vp, i64, ctypes.c_double, ctypes.POINTER(CsrOut), ctypes.POINTER(i64),
                                            ctypes.POINTER(RequestInfo)]
        lib.gbla_server_wait_ex.restype = i32
        lib.gbla_server_poll.argtypes = [vp, i64, ctypes.POINTER(i32)]
        lib.gbla_server_poll.restype = i32
        lib.gbla_server_cancel.argtypes = [vp, i64]
        lib.gbla_server_cancel.restype = i32
        lib.gbla_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
        lib.gbla_server_get_stats.restype = i32
        lib.gbla_server_destroy.argtypes = [vp]
        lib.gbla_server_destroy.restype = None
        lib.gbla_decode_format2.argtypes = [ctypes.c_char_p, ctypes.c_size_t, vp, ctypes.POINTER(CsrOut),
                                            ctypes.POINTER(u32)]
        lib.gbla_decode_format2.restype = i32
        lib.gbla_decode_format2_ex.argtypes = [vp, ctypes.c_size_t, vp, ctypes.POINTER(CsrOut),
                                               ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_double)]
        lib.gbla_decode_format2_ex.restype = i32
        _lib = lib
        return lib


def strerror(code: int) -> str:
    try:
        return load().gbla_strerror(code).decode()
    except Exception:  # library missing: still give a message
        return "error"


def _check(rc, what):
    if rc != GBLA_OK:
        raise GblaError(rc, what)


def _stream_ptr(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


class HostResult:
    """A result in the library's page-locked host memory.  ``row_ptr``,
    ``col`` and ``val`` are zero-copy numpy views, valid until free()."""

    def __init__(self, out: CsrOut, rank: int, stats: dict):
        self._out = out
        self.rank = rank
        self.nnz = int(out.nnz)
        self.stats = stats
        self.row_ptr = np.ctypeslib.as_array(ctypes.cast(out.row_ptr, ctypes.POINTER(ctypes.c_int64)),
                                             shape=(rank + 1,))
        if self.nnz:
            self.col = np.ctypeslib.as_array(ctypes.cast(out.col, ctypes.POINTER(ctypes.c_int32)), shape=(self.nnz,))
            self.val = np.ctypeslib.as_array(ctypes.cast(out.val, ctypes.POINTER(ctypes.c_uint16)), shape=(self.nnz,))
        else:
            self.col = np.zeros(0, np.int32)
            self.val = np.zeros(0, np.uint16)

    def free(self):
        if self._out is not None:
            self.row_ptr = self.col = self.val = None
            load().gbla_free(ctypes.byref(self._out))
            self._out = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def reduce_host(row_ptr, col, val, shape, p, want_reduced=False, variant=GEMM_AUTO, stream=None,
                path=PATH_AUTO, leaf=0, order=ORDER_NEW, autotune=False, echelon=ECHELON_AUTO) -> HostResult:
    """Reduce a host CSR matrix; the result stays in library-owned host memory
    (see HostResult).  Page-locked inputs copy to the device fastest.
    ``path`` is PATH_AUTO, PATH_DENSE or PATH_SPARSE, ``leaf`` the leaf width
    of the triangular solve (0 = chosen per matrix)."""
    lib = load()
    m, n = int(shape[0]), int(shape[1])
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.uint16)
    cin = CsrIn(m, n, int(len(col)), row_ptr.ctypes.data, col.ctypes.data, val.ctypes.data)
    opt = _options(want_reduced, variant, 0, path, leaf, order=order, autotune=autotune, echelon=echelon)
    out = CsrOut()
    rank = ctypes.c_int64(0)
    st = Stats()
    rc = lib.gbla_reduce_ex(ctypes.byref(cin), int(p), ctypes.byref(opt), _stream_ptr(stream),
                            ctypes.byref(out), ctypes.byref(rank), ctypes.byref(st))
    _check(rc, "gbla_reduce_ex")
    return HostResult(out, int(rank.value), st.as_dict())


def reduce(row_ptr, col, val, shape, p, want_reduced=False, variant=GEMM_AUTO, stats=False, stream=None,
           path=PATH_AUTO, leaf=0, order=ORDER_NEW, autotune=False, echelon=ECHELON_AUTO):
    """Reduce a host CSR matrix.  Returns (rank, row_ptr, col, val) as numpy
    arrays the caller owns (and a stats dict when ``stats``)."""
    h = reduce_host(row_ptr, col, val, shape, p, want_reduced=want_reduced, variant=variant, stream=stream,
                    path=path, leaf=leaf, order=order, autotune=autotune, echelon=echelon)
    try:
        res = (h.rank, h.row_ptr.copy(), h.col.copy(), h.val.copy())
        st = h.stats
    finally:
        h.free()
    return res + (st,) if stats else res


class DeviceResult:
    """A result left in device memory (owned by the library until free())."""

    def __init__(self, out: CsrOut, rank: int, stats: dict):
        self._out = out
        self.rank = rank
        self.nnz = int(out.nnz)
        self.stats = stats

    def tensors(self):
        """Zero-copy torch views (row_ptr, col, val) of the device arrays;
        valid until free()."""
        import torch
        r, nnz = self.rank, self.nnz
        rp = torch.as_tensor(_CudaArray(self._out.row_ptr, (r + 1,), "<i8"), device="cuda")
        oc = torch.as_tensor(_CudaArray(self._out.col, (nnz,), "<i4"), device="cuda")
        ov = torch.as_tensor(_CudaArray(self._out.val, (nnz,), "<i2"), device="cuda")
        return rp, oc, ov

    def to_host(self):
        rp, oc, ov = self.tensors()
        return (self.rank, rp.cpu().numpy(), oc.cpu().numpy(),
                ov.cpu().numpy().view(np.uint16))

    def free(self):
        if self._out is not None:
            load().gbla_free(ctypes.byref(self._out))
            self._out = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class DecodedMatrix(DeviceResult):
    """A matrix decoded on the device (owned by the library until free()):
    m x n over GF(p); tensors() gives its row_ptr, col and val, the input
    form of reduce_device."""

    def __init__(self, out: CsrOut, p: int):
        super().__init__(out, int(out.nrows), {})
        self.m, self.n, self.p = int(out.nrows), int(out.ncols), int(p)


def decode_format2(buf, stream=None, timed=False) -> DecodedMatrix:
    """Decode a Format 2 matrix file (bytes, or a contiguous uint8 numpy
    array such as a page-locked buffer; Sec. 3.2 of the paper) on the
    device; raises GblaError (GBLA_E_INVAL) on a malformed file.  With
    timed=True the result's ``decode_ms`` is the event-timed device work of
    the decode (host-to-device copies excluded)."""
    lib = load()
    if isinstance(buf, np.ndarray):
        assert buf.dtype == np.uint8 and buf.flags["C_CONTIGUOUS"]
        keep, ptr, nbytes = buf, ctypes.c_void_p(buf.ctypes.data), buf.nbytes
    else:
        keep = bytes(buf)
        ptr, nbytes = ctypes.cast(ctypes.c_char_p(keep), ctypes.c_void_p), len(keep)
    out = CsrOut()
    p = ctypes.c_uint32(0)
    ms = ctypes.c_double(-1.0)
    rc = lib.gbla_decode_format2_ex(ptr, nbytes, _stream_ptr(stream), ctypes.byref(out), ctypes.byref(p),
                                    ctypes.byref(ms) if timed else None)
    del keep
    _check(rc, "gbla_decode_format2")
    d = DecodedMatrix(out, p.value)
    d.decode_ms = float(ms.value) if timed else None
    return d


class _CudaArray:
    """Minimal __cuda_array_interface__ over a raw device pointer."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr,
                                         "data": (int(ptr or 0), False), "version": 3, "strides": None}


def reduce_device(row_ptr, col, val, shape, p, want_reduced=False, variant=GEMM_AUTO, stream=None,
                  path=PATH_AUTO, leaf=0, kernel_times=False, order=ORDER_NEW, autotune=False,
                  echelon=ECHELON_AUTO):
    """Reduce a CSR matrix already on the device (torch CUDA tensors: int64
    row_ptr, int32 col, int16/uint16 val).  Returns a DeviceResult whose
    arrays stay in device memory."""
    lib = load()
    m, n = int(shape[0]), int(shape[1])
    cin = CsrIn(m, n, int(col.numel()), row_ptr.data_ptr(), col.data_ptr(), val.data_ptr())
    opt = _options(want_reduced, variant, 1, path, leaf, kernel_times, order, autotune, echelon)
    out = CsrOut()
    rank = ctypes.c_int64(0)
    st = Stats()
    rc = lib.gbla_reduce_ex(ctypes.byref(cin), int(p), ctypes.byref(opt), _stream_ptr(stream),
                            ctypes.byref(out), ctypes.byref(rank), ctypes.byref(st))
    _check(rc, "gbla_reduce_ex")
    return DeviceResult(out, int(rank.value), st.as_dict())


def _host_result(lib, out):
    """Copy a host gbla_csr_out into numpy arrays and release it."""
    try:
        r = int(out.nrows)
        onnz = int(out.nnz)
        orp = np.ctypeslib.as_array(ctypes.cast(out.row_ptr, ctypes.POINTER(ctypes.c_int64)), shape=(r + 1,)).copy()
        if onnz:
            oc = np.ctypeslib.as_array(ctypes.cast(out.col, ctypes.POINTER(ctypes.c_int32)), shape=(onnz,)).copy()
            ov = np.ctypeslib.as_array(ctypes.cast(out.val, ctypes.POINTER(ctypes.c_uint16)), shape=(onnz,)).copy()
        else:
            oc = np.zeros(0, np.int32)
            ov = np.zeros(0, np.uint16)
    finally:
        lib.gbla_free(ctypes.byref(out))
    return orp, oc, ov


def _csr_in(row_ptr, col, val, shape):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.uint16)
    cin = CsrIn(int(shape[0]), int(shape[1]), int(len(col)), row_ptr.ctypes.data, col.ctypes.data,
                val.ctypes.data)
    return cin, (row_ptr, col, val)


def reduce_batch(mats, want_reduced=False, variant=GEMM_AUTO, workers=0, path=PATH_AUTO, autotune=False):
    """Reduce many host CSR matrices on a pool of worker threads whose
    reductions overlap on the device.  ``mats`` is a list of
    (row_ptr, col, val, shape, p).  Returns a list of (rank, row_ptr, col, val)
    (raises on the first failure)."""
    lib = load()
    n = len(mats)
    keep = []
    ins = (CsrIn * max(n, 1))()
    ps = (ctypes.c_uint32 * max(n, 1))()
    for i, (rp, c, v, shape, p) in enumerate(mats):
        cin, arrs = _csr_in(rp, c, v, shape)
        keep.append(arrs)
        ins[i] = cin
        ps[i] = int(p)
    opt = _options(want_reduced, variant, 0, path, autotune=autotune)
    outs = (CsrOut * max(n, 1))()
    ranks = (ctypes.c_int64 * max(n, 1))()
    codes = (ctypes.c_int * max(n, 1))()
    rc = lib.gbla_reduce_batch(n, ins, ps, ctypes.byref(opt), int(workers), outs, ranks, codes)
    res = []
    for i in range(n):
        if codes[i] == GBLA_OK:
            res.append((int(ranks[i]),) + _host_result(lib, outs[i]))
        else:
            lib.gbla_free(ctypes.byref(outs[i]))
            res.append(None)
    _check(rc, "gbla_reduce_batch")
    return res


def reduce_batch_device(mats, want_reduced=False, variant=GEMM_AUTO, workers=0, path=PATH_AUTO,
                        autotune=False):
    """Reduce many matrices already on the device through the batch entry
    point (workers whose reductions overlap on the device).  ``mats`` is a
    list of (row_ptr, col, val, shape, p) with int64 / int32 / 16-bit CUDA
    tensors.  Returns a list of DeviceResult (raises on the first failure)."""
    lib = load()
    n = len(mats)
    ins = (CsrIn * max(n, 1))()
    ps = (ctypes.c_uint32 * max(n, 1))()
    for i, (rp, c, v, shape, p) in enumerate(mats):
        ins[i] = CsrIn(int(shape[0]), int(shape[1]), int(c.numel()), rp.data_ptr(), c.data_ptr(), v.data_ptr())
        ps[i] = int(p)
    opt = _options(want_reduced, variant, 1, path, autotune=autotune)
    outs = (CsrOut * max(n, 1))()
    ranks = (ctypes.c_int64 * max(n, 1))()
    codes = (ctypes.c_int * max(n, 1))()
    rc = lib.gbla_reduce_batch(n, ins, ps, ctypes.byref(opt), int(workers), outs, ranks, codes)
    res = [DeviceResult(outs[i], int(ranks[i]), {}) for i in range(n)]
    if rc != GBLA_OK:
        for r in res:
            r.free()
    _check(rc, "gbla_reduce_batch")
    return res


class Server:
    """Request server with continuous batching (see gbla_server_* in gbla.h)."""

    def __init__(self, mem_budget=0, workers=0):
        self._lib = load()
        self._h = ctypes.c_void_p()
        _check(self._lib.gbla_server_create(int(mem_budget), int(workers), ctypes.byref(self._h)),
               "gbla_server_create")

    def submit(self, row_ptr, col, val, shape, p, want_reduced=False, variant=GEMM_AUTO, path=PATH_AUTO,
               autotune=False):
        cin, _arrs = _csr_in(row_ptr, col, val, shape)   # copied by the server at submit
        opt = _options(want_reduced, variant, 0, path, autotune=autotune)
        t = ctypes.c_int64(0)
        _check(self._lib.gbla_server_submit(self._h, ctypes.byref(cin), int(p), ctypes.byref(opt), ctypes.byref(t)),
               "gbla_server_submit")
        return int(t.value)

    def wait(self, ticket, timeout=-1.0):
        """Returns (code, result or None, latency_ms)."""
        out = CsrOut()
        rank = ctypes.c_int64(0)
        lat = ctypes.c_double(0)
        rc = self._lib.gbla_server_wait(self._h, int(ticket), float(timeout), ctypes.byref(out),
                                        ctypes.byref(rank), ctypes.byref(lat))
        if rc == GBLA_OK:
            return rc, (int(rank.value),) + _host_result(self._lib, out), float(lat.value)
        self._lib.gbla_free(ctypes.byref(out))
        return rc, None, float(lat.value)

    def wait_ex(self, ticket, timeout=-1.0):
        """Returns (code, result or None, timeline dict: latency_ms, queue_ms,
        device_start_ms, device_end_ms, running_at_start)."""
        out = CsrOut()
        rank = ctypes.c_int64(0)
        info = RequestInfo()
        rc = self._lib.gbla_server_wait_ex(self._h, int(ticket), float(timeout), ctypes.byref(out),
                                           ctypes.byref(rank), ctypes.byref(info))
        if rc == GBLA_OK:
            return rc, (int(rank.value),) + _host_result(self._lib, out), info.as_dict()
        self._lib.gbla_free(ctypes.byref(out))
        return rc, None, info.as_dict()

    def poll(self, ticket):
        """REQ_QUEUED, REQ_RUNNING, REQ_DONE or REQ_CANCELLED (raises for an
        unknown or consumed ticket)."""
        st = ctypes.c_int(-1)
        _check(self._lib.gbla_server_poll(self._h, int(ticket), ctypes.byref(st)), "gbla_server_poll")
        return int(st.value)

    def cancel(self, ticket):
        return int(self._lib.gbla_server_cancel(self._h, int(ticket)))

    def stats(self):
        st = ServerStats()
        _check(self._lib.gbla_server_get_stats(self._h, ctypes.byref(st)), "gbla_server_get_stats")
        return st.as_dict()

    def close(self):
        if self._h:
            self._lib.gbla_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def modmatmul(A, B, C, p, sign=-1, variant=GEMM_AUTO, stream=None):
    """C <- (C + sign*A*B) mod p in place; A, B, C are 2-D row-major CUDA
    tensors of 16-bit values (int16 views of uint16 residues)."""
    lib = load()
    M, K = A.shape
    K2, N = B.shape
    assert K2 == K and tuple(C.shape) == (M, N)
    rc = lib.gbla_modmatmul(M, N, K, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0),
                            C.data_ptr(), C.stride(0), int(p), int(sign), int(variant), _stream_ptr(stream))
    _check(rc, "gbla_modmatmul")


def fail_alloc_after(n):
    """Arm the one-shot allocation fault: the allocation after the next n
    fails (n < 0 disarms).  Test hook."""
    _check(load().gbla_selftest_fail_alloc_after(int(n)), "gbla_selftest_fail_alloc_after")


def device_bytes_in_use():
    """Bytes of the device pool held by the library (synchronises the device)."""
    v = ctypes.c_int64(0)
    _check(load().gbla_device_bytes_in_use(ctypes.byref(v)), "gbla_device_bytes_in_use")
    return int(v.value)


def pipe_peak(variant, stream=None):
    """Measured issue rate (1e12 ops/s) of the FP64 or U8 mma.sync pipe."""
    lib = load()
    out = ctypes.c_double(0.0)
    _check(lib.gbla_pipe_peak(int(variant), ctypes.byref(out), _stream_ptr(stream)), "gbla_pipe_peak")
    return out.value


def modmatmul32(A, B, C, p, sign=-1, stream=None):
    """C <- (C + sign*A*B) mod p in place for a prime p < 2^31; A, B, C are 2-D
    row-major CUDA tensors of 32-bit values (int32 views of uint32 residues)."""
    lib = load()
    M, K = A.shape
    K2, N = B.shape
    assert K2 == K and tuple(C.shape) == (M, N)
    rc = lib.gbla_modmatmul32(M, N, K, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0),
                              C.data_ptr(), C.stride(0), int(p), int(sign), _stream_ptr(stream))
    _check(rc, "gbla_modmatmul32")


def spmm(X, S_row_ptr, S_col, S_val, N, C, p, sign=-1, x_lead=None, stream=None):
    """C <- (C + sign * X * S) mod p in place: X (M x K) and C (M x N) 2-D
    row-major CUDA tensors of 16-bit values, S a K x N CSR matrix given by
    CUDA tensors (int64 row_ptr, int32 col, 16-bit val); x_lead an optional
    int32 CUDA tensor of ascending row leads of X.  Runs the K-compacted
    tensor-core product of the sparse path."""
    lib = load()
    M, K = X.shape
    cin = CsrIn(K, int(N), int(S_col.numel()), S_row_ptr.data_ptr(), S_col.data_ptr(), S_val.data_ptr())
    rc = lib.gbla_spmm(M, int(N), K, X.data_ptr(), X.stride(0), ctypes.byref(cin),
                       None if x_lead is None else x_lead.data_ptr(), C.data_ptr(), C.stride(0), int(p),
                       int(sign), _stream_ptr(stream))
    _check(rc, "gbla_spmm")


def pivots(row_ptr, col, val, shape, p, stream=None):
    """FL step-1 pivot choice on device tensors; returns (piv_row tensor, npiv)."""
    import torch
    lib = load()
    m, n = int(shape[0]), int(shape[1])
    cin = CsrIn(m, n, int(col.numel()), row_ptr.data_ptr(), col.data_ptr(), val.data_ptr())
    out = torch.empty(max(n, 1), dtype=torch.int64, device=row_ptr.device)
    npiv = ctypes.c_int64(0)
    rc = lib.gbla_pivots(ctypes.byref(cin), int(p), out.data_ptr(), ctypes.byref(npiv), _stream_ptr(stream))
    _check(rc, "gbla_pivots")
    return out[:n], int(npiv.value)


def _check_noalloc_args(row_ptr, col, val, m, n, out):
    """The library writes n int64 values through ``out`` and reads the CSR
    through the other pointers without knowing their sizes, so every tensor
    is checked here: contiguous CUDA tensors of the right type and length,
    all on one device."""
    import torch
    named = (("row_ptr", row_ptr, (torch.int64,)), ("col", col, (torch.int32,)),
             ("val", val, (torch.int16, getattr(torch, "uint16", torch.int16))), ("out", out, (torch.int64,)))
    for name, t, dtypes in named:
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if t.dtype not in dtypes:
            raise ValueError(f"{name} has dtype {t.dtype}, expected {dtypes[0]}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if m < 0 or n < 0:
        raise ValueError("negative shape")
    if row_ptr.numel() != m + 1:
        raise ValueError(f"row_ptr has {row_ptr.numel()} entries, expected m + 1 = {m + 1}")
    if val.numel() != col.numel():
        raise ValueError("col and val differ in length")
    if out.numel() < n:
        raise ValueError(f"out has {out.numel()} entries, expected at least ncols = {n}")
    for name, t, _ in named:
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.device != out.device:
            raise ValueError(f"{name} is on {t.device}, out on {out.device}")


def pivots_noalloc(row_ptr, col, val, shape, p, out, stream=None):
    """Pivot choice without any allocation in the library: writes piv_row into
    the caller's int64 CUDA tensor ``out`` (at least ncols long) and returns
    npiv.  For callers that must not allocate device memory during a call;
    at most 2^20 columns; calls that overlap on the GPU race.  The tensors
    are checked (ValueError) before the library sees them; the call runs with
    ``out``'s device current."""
    import torch
    m, n = int(shape[0]), int(shape[1])
    _check_noalloc_args(row_ptr, col, val, m, n, out)
    lib = load()
    cin = CsrIn(m, n, int(col.numel()), row_ptr.data_ptr(), col.data_ptr(), val.data_ptr())
    npiv = ctypes.c_int64(0)
    with torch.cuda.device(out.device):
        rc = lib.gbla_pivots_noalloc(ctypes.byref(cin), int(p), out.data_ptr(), ctypes.byref(npiv),
                                     _stream_ptr(stream))
    _check(rc, "gbla_pivots_noalloc")
    return int(npiv.value)


def selftest_wait_timeout(stream=None) -> int:
    """Run one product tile whose loads are withheld; returns the status code
    (GBLA_E_TIMEOUT = 4 expected: the bounded waits expired and the kernel
    returned cleanly)."""
    return int(load().gbla_selftest_wait_timeout(_stream_ptr(stream)))


def multiline(row_ptr, col, val, m):
    """2-multiline vectors of consecutive row pairs of a host CSR (computed on
    the device).  Returns (ml_ptr, ml_pos, ml_val) numpy arrays."""
    lib = load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.uint16)
    nnz = len(col)
    cin = CsrIn(m, 0, nnz, row_ptr.ctypes.data, col.ctypes.data, val.ctypes.data)
    npairs = (m + 1) // 2
    ptr = np.zeros(npairs + 1, np.int64)
    pos = np.zeros(max(nnz, 1), np.int32)
    mv = np.zeros(max(2 * nnz, 2), np.uint16)
    rc = lib.gbla_multiline(ctypes.byref(cin), ptr.ctypes.data, pos.ctypes.data, mv.ctypes.data, None)
    _check(rc, "gbla_multiline")
    total = int(ptr[-1])
    return ptr, pos[:total], mv[:2 * total]
