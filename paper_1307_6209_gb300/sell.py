"""Thin Python binding of the SELL-C-sigma C ABI (include/sell.h).

Argument marshalling only: every step of the computation runs in the CUDA
library ``_build/libsellcs.so``.  Device buffers are torch tensors (or raw
device pointers); host buffers are numpy arrays.  The names follow the C
entry points.  There is no fallback: if the library is missing, ``load()``
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsellcs.so")

SELL_F64, SELL_F32, SELL_BF16 = 0, 1, 2
SELL_OK, SELL_EINVAL, SELL_ENOMEM, SELL_ECUDA, SELL_EBOUNDS, SELL_ETIMEOUT, SELL_EUNSUPPORTED = range(7)
SELL_BUILD_PERMUTE_COLS = 0x1
SELL_SPMV_ACCUMULATE = 0x1
SELL_SPMV_COMPENSATED = 0x2
SELL_SPMV_HOST_IO = 0x4
SELL_SPMV_COMPENSATED_LONG = 0x8
SELL_SPMV_HOST_DIRECT = 0x80
SELL_SPMV_RHS_BLOCK4 = 0x10
SELL_SPMV_RHS_BLOCK2 = 0x20
SELL_SPMV_RHS_BLOCK1 = 0x40

DTYPE_NAMES = {SELL_F64: "f64", SELL_F32: "f32", SELL_BF16: "bf16"}
VALUE_BYTES = {SELL_F64: 8, SELL_F32: 4, SELL_BF16: 2}


class SellError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"sell status {status}: {msg}")
        self.status = status


class sell_csr(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rpt", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("val_type", ctypes.c_int32), ("on_device", ctypes.c_int32)]


class sell_opts(ctypes.Structure):
    _fields_ = [("C", ctypes.c_int32), ("store_type", ctypes.c_int32), ("sigma", ctypes.c_int64),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_int32)]


class sell_info_t(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("nchunks", ctypes.c_int64), ("stored", ctypes.c_int64),
                ("max_row_len", ctypes.c_int64), ("sigma", ctypes.c_int64), ("C", ctypes.c_int32),
                ("store_type", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("has_perm", ctypes.c_int32), ("beta", ctypes.c_double), ("zeta", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t)]


class sell_batch_item(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("X", ctypes.c_void_p), ("Y", ctypes.c_void_p),
                ("ldx", ctypes.c_int64), ("ldy", ctypes.c_int64), ("k", ctypes.c_int32),
                ("flags", ctypes.c_uint32)]


class sell_server_opts(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("max_batch", ctypes.c_int32), ("streams", ctypes.c_int32),
                ("size_ratio", ctypes.c_int32), ("reserved", ctypes.c_int32), ("max_batch_work", ctypes.c_int64)]


class sell_request_info(ctypes.Structure):
    _fields_ = [("t_arrive", ctypes.c_double), ("t_launch", ctypes.c_double), ("t_done", ctypes.c_double),
                ("batch", ctypes.c_int32), ("status", ctypes.c_int32)]


class sell_server_stats_t(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_int64), ("batches", ctypes.c_int64), ("batched_requests", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("resident_bytes", ctypes.c_int64), ("budget_bytes", ctypes.c_int64),
                ("in_use_bytes", ctypes.c_int64), ("peak_bytes", ctypes.c_int64)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

# every exported entry point with (restype, argtypes)
_P = ctypes.c_void_p
SIGNATURES = {
    "sell_set_allocator": (ctypes.c_int, [ALLOC_FN, FREE_FN, _P]),
    "sell_build": (ctypes.c_int, [ctypes.POINTER(sell_csr), ctypes.POINTER(sell_opts), _P,
                                  ctypes.POINTER(_P)]),
    "sell_spmv": (ctypes.c_int, [_P, _P, _P, ctypes.c_uint32, _P]),
    "sell_spmmv": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_int32,
                                  ctypes.c_uint32, _P]),
    "sell_spmv_dot": (ctypes.c_int, [_P, _P, _P, ctypes.c_uint32, _P, _P]),
    "sell_spmmv_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_int32,
                                          ctypes.c_uint32, _P]),
    "sell_set_launch": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "sell_check": (ctypes.c_int, [_P, _P]),
    "sell_test_expire_wait": (ctypes.c_int, [_P, ctypes.c_uint32]),
    "sell_info": (ctypes.c_int, [_P, ctypes.POINTER(sell_info_t)]),
    "sell_export": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "sell_free": (ctypes.c_int, [_P]),
    "sell_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "sell_last_error": (ctypes.c_char_p, []),
    "sell_batch_create": (ctypes.c_int, [ctypes.POINTER(sell_batch_item), ctypes.c_int32, _P,
                                         ctypes.POINTER(_P)]),
    "sell_batch_run": (ctypes.c_int, [_P, ctypes.c_int32, _P]),
    "sell_batch_free": (ctypes.c_int, [_P]),
    "sell_batch_set_launch": (ctypes.c_int, [_P, ctypes.c_int32]),
    "sell_server_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, ctypes.POINTER(sell_server_opts),
                                          ctypes.POINTER(_P)]),
    "sell_server_submit": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32, _P, ctypes.c_uint32,
                                          ctypes.POINTER(ctypes.c_uint64)]),
    "sell_server_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(sell_request_info)]),
    "sell_server_next": (ctypes.c_int, [_P, ctypes.c_double, ctypes.POINTER(ctypes.c_uint64),
                                        ctypes.POINTER(sell_request_info)]),
    "sell_server_result": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(_P)]),
    "sell_server_release": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "sell_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(sell_server_stats_t)]),
    "sell_server_destroy": (ctypes.c_int, [_P]),
    "sell_bench_read": (ctypes.c_int, [_P, ctypes.c_size_t, _P, ctypes.c_int32, _P]),
    "sell_bench_fma64": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P]),
    "sell_bench_gather": (ctypes.c_int, [_P, ctypes.c_int64, _P, ctypes.c_int32, ctypes.c_int32, _P]),
    "sell_bench_gather4": (ctypes.c_int, [_P, ctypes.c_int64, _P, ctypes.c_int32, ctypes.c_int32, _P]),
}

_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"SELL CUDA library not built: {p} is missing "
                               "(run __graft_entry__.build() or paper_1307_6209_gb300/build.py)")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(st):
    if st != SELL_OK:
        lib = load()
        raise SellError(st, lib.sell_last_error().decode())


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    """Address of a torch tensor or numpy array (or an int address)."""
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    if isinstance(t, np.ndarray):
        return ctypes.c_void_p(t.ctypes.data)
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ handle
@dataclass
class Info:
    nrows: int
    ncols: int
    nnz: int
    nchunks: int
    stored: int
    max_row_len: int
    sigma: int
    C: int
    store_type: int
    flags: int
    has_perm: bool
    beta: float
    zeta: float
    device_bytes: int


class SellMatrix:
    """Owns a ``sell_handle``; freed with ``sell_free`` (or on garbage collection)."""

    def __init__(self, handle: int, keepalive=None):
        self.handle = ctypes.c_void_p(handle)
        self._keep = keepalive
        self.info = sell_info(self)

    def free(self):
        if self.handle and self.handle.value:
            _check(load().sell_free(self.handle))
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def value_dtype(self):
        import torch
        return torch.float64 if self.info.store_type == SELL_F64 else torch.float32


def sell_build(A, C: int = 32, sigma: int = 1, store_type: int = SELL_F64, flags: int = 0,
               stream=None) -> SellMatrix:
    """Build a SELL-C-sigma handle from a CSR matrix.  ``A`` has nrows, ncols,
    rpt, col, val; numpy arrays are host CRS, torch CUDA tensors device CRS."""
    lib = load()
    rpt, col, val = A.rpt, A.col, A.val
    keep = []
    if isinstance(rpt, np.ndarray):
        rpt = np.ascontiguousarray(rpt, np.int64)
        col = np.ascontiguousarray(col, np.int32)
        if val.dtype not in (np.float64, np.float32):
            val = val.astype(np.float64)
        val = np.ascontiguousarray(val)
        on_device = 0
        vt = SELL_F64 if val.dtype == np.float64 else SELL_F32
    else:
        import torch
        assert rpt.is_cuda and rpt.dtype == torch.int64 and col.dtype == torch.int32
        on_device = 1
        vt = SELL_F64 if val.dtype == torch.float64 else SELL_F32
        rpt, col, val = rpt.contiguous(), col.contiguous(), val.contiguous()
    keep += [rpt, col, val]
    nnz = int(rpt[-1]) if A.nrows > 0 else 0
    csr = sell_csr(int(A.nrows), int(A.ncols), nnz, _ptr(rpt), _ptr(col), _ptr(val), vt, on_device)
    opts = sell_opts(int(C), int(store_type), int(sigma), int(flags), 0)
    out = ctypes.c_void_p()
    _check(lib.sell_build(ctypes.byref(csr), ctypes.byref(opts), _stream_ptr(stream), ctypes.byref(out)))
    return SellMatrix(out.value)


def _check_vec(h: SellMatrix, t, name: str, host: bool, rows: bool = True):
    """The element type and placement the C call expects (binary64 for F64
    handles, binary32 otherwise; device memory unless host I/O; unit stride
    along the right-hand sides)."""
    if t is None or isinstance(t, int):
        return
    want64 = h.info.store_type == SELL_F64
    if isinstance(t, np.ndarray):
        ok = t.dtype == (np.float64 if want64 else np.float32)
        if not ok:
            raise TypeError(f"{name}: expected {'float64' if want64 else 'float32'}, got {t.dtype}")
        if not host:
            raise TypeError(f"{name}: a numpy array needs SELL_SPMV_HOST_IO or SELL_SPMV_HOST_DIRECT")
        inner = t.strides[-1] // t.itemsize if t.ndim > 1 else 1
    else:
        import torch
        if t.dtype != (torch.float64 if want64 else torch.float32):
            raise TypeError(f"{name}: expected {'float64' if want64 else 'float32'}, got {t.dtype}")
        if t.is_cuda == host:
            raise TypeError(f"{name}: {'host' if host else 'device'} memory expected")
        inner = t.stride(-1) if t.dim() > 1 else t.stride(0)
    if inner != 1:
        raise ValueError(f"{name}: the right-hand sides must be contiguous in each row (unit inner stride)")


def sell_spmv(h: SellMatrix, x, y, flags: int = 0, stream=None):
    host = bool(int(flags) & (SELL_SPMV_HOST_IO | SELL_SPMV_HOST_DIRECT))
    _check_vec(h, x, "x", host)
    _check_vec(h, y, "y", host)
    _check(load().sell_spmv(h.handle, _ptr(x), _ptr(y), int(flags), _stream_ptr(stream)))
    return y


def sell_spmv_dot(h: SellMatrix, x, y, dot, flags: int = 0, stream=None):
    """y = A x, then dot[0] = x . y (binary64, fixed summation order); dot is a
    device float64 tensor of at least one element."""
    _check(load().sell_spmv_dot(h.handle, _ptr(x), _ptr(y), int(flags), _ptr(dot), _stream_ptr(stream)))


def sell_spmmv(h: SellMatrix, X, Y, flags: int = 0, stream=None, ldx=None, ldy=None, k=None):
    """Y = A X for row-major X (ncols x k) and Y (nrows x k)."""
    host = bool(int(flags) & (SELL_SPMV_HOST_IO | SELL_SPMV_HOST_DIRECT))
    _check_vec(h, X, "X", host)
    _check_vec(h, Y, "Y", host)
    k = int(X.shape[1]) if k is None else int(k)
    ldx = int(X.stride(0) if hasattr(X, "stride") and callable(X.stride) else X.strides[0] // X.itemsize) \
        if ldx is None else int(ldx)
    ldy = int(Y.stride(0) if hasattr(Y, "stride") and callable(Y.stride) else Y.strides[0] // Y.itemsize) \
        if ldy is None else int(ldy)
    _check(load().sell_spmmv(h.handle, _ptr(X), ldx, _ptr(Y), ldy, k, int(flags), _stream_ptr(stream)))
    return Y


def sell_spmmv_noalloc(h: SellMatrix, X, Y, flags: int = 0, stream=None):
    """Y = A X like sell_spmmv, allocating nothing (long-row scratch in the
    library's fixed 4 MiB device array; see include/sell.h)."""
    if X.dim() == 1:
        k, ldx, ldy = 1, 1, 1
    else:
        k, ldx, ldy = int(X.shape[1]), int(X.stride(0)), int(Y.stride(0))
    _check(load().sell_spmmv_noalloc(h.handle, _ptr(X), ldx, _ptr(Y), ldy, k, int(flags), _stream_ptr(stream)))
    return Y


def sell_set_launch(h: SellMatrix, block: int = 0, unroll: int = 0, pipeline: int = -1):
    """Launch shape of the handle's kernels (0 / -1 keep the current value)."""
    _check(load().sell_set_launch(h.handle, int(block), int(unroll), int(pipeline)))


def sell_check(h: SellMatrix, stream=None):
    """Synchronise the stream; raise SellError(SELL_ETIMEOUT) if a bounded
    device-side wait of the handle's kernels gave up."""
    _check(load().sell_check(h.handle, _stream_ptr(stream)))


def sell_test_expire_wait(h: SellMatrix, limit_us: int):
    """Test hook: the next bulk-staged product's first warp waits limit_us on
    a barrier nothing completes, so sell_check then reports SELL_ETIMEOUT."""
    _check(load().sell_test_expire_wait(h.handle, int(limit_us)))


def sell_info(h: SellMatrix) -> Info:
    inf = sell_info_t()
    _check(load().sell_info(h.handle, ctypes.byref(inf)))
    return Info(inf.nrows, inf.ncols, inf.nnz, inf.nchunks, inf.stored, inf.max_row_len, inf.sigma,
                inf.C, inf.store_type, inf.flags, bool(inf.has_perm), inf.beta, inf.zeta,
                inf.device_bytes)


def sell_export(h: SellMatrix) -> dict:
    """Host copies of the format arrays (val as float64/float32/uint16 bits)."""
    inf = h.info
    vdt = {SELL_F64: np.float64, SELL_F32: np.float32, SELL_BF16: np.uint16}[inf.store_type]
    val = np.empty(inf.stored, vdt)
    col = np.empty(inf.stored, np.int32)
    cs = np.empty(inf.nchunks + 1, np.int64)
    cl = np.empty(inf.nchunks, np.int32)
    rl = np.empty(inf.nchunks * inf.C, np.int32)
    perm = np.empty(inf.nrows, np.int32)
    _check(load().sell_export(h.handle, _ptr(val), _ptr(col), _ptr(cs), _ptr(cl), _ptr(rl), _ptr(perm)))
    return {"val": val, "col": col, "cs": cs, "cl": cl, "srl": rl, "perm": perm}


def sell_free(h: SellMatrix):
    h.free()


def sell_strerror(status: int) -> str:
    return load().sell_strerror(int(status)).decode()


def sell_last_error() -> str:
    return load().sell_last_error().decode()


# ------------------------------------------------------------------ batching
class BatchPlan:
    def __init__(self, handle: int, keepalive):
        self.handle = ctypes.c_void_p(handle)
        self._keep = keepalive

    def run(self, grid: int = 0, stream=None):
        _check(load().sell_batch_run(self.handle, int(grid), _stream_ptr(stream)))

    def set_launch(self, block: int):
        """Threads per block (64, 128, 256): rows per work unit."""
        _check(load().sell_batch_set_launch(self.handle, int(block)))

    def free(self):
        if self.handle and self.handle.value:
            _check(load().sell_batch_free(self.handle))
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sell_batch_create(items, stream=None) -> BatchPlan:
    """items: iterable of (SellMatrix, X, Y, flags) with X (ncols x k) and Y
    (nrows x k) row-major torch tensors, or 1-D vectors for k = 1."""
    arr = (sell_batch_item * max(1, len(items)))()
    keep = []
    for i, (h, X, Y, fl) in enumerate(items):
        if X.dim() == 1:
            k, ldx, ldy = 1, 1, 1
        else:
            k, ldx, ldy = int(X.shape[1]), int(X.stride(0)), int(Y.stride(0))
        arr[i] = sell_batch_item(h.handle.value, X.data_ptr(), Y.data_ptr(), ldx, ldy, k, int(fl))
        keep.append((h, X, Y))
    out = ctypes.c_void_p()
    _check(load().sell_batch_create(arr, len(items), _stream_ptr(stream), ctypes.byref(out)))
    return BatchPlan(out.value, keep)


def sell_batch_run(plan: BatchPlan, grid: int = 0, stream=None):
    plan.run(grid, stream)


def sell_batch_free(plan: BatchPlan):
    plan.free()


# ------------------------------------------------------------------ measuring
def sell_bench_read(buf, nbytes: int, sink, grid: int = 0, stream=None):
    _check(load().sell_bench_read(_ptr(buf), int(nbytes), _ptr(sink), int(grid), _stream_ptr(stream)))


def sell_bench_gather(x, n: int, sink, grid: int, iters: int, stream=None):
    _check(load().sell_bench_gather(_ptr(x), int(n), _ptr(sink), int(grid), int(iters), _stream_ptr(stream)))


def sell_bench_gather4(x, n: int, sink, grid: int, iters: int, stream=None):
    _check(load().sell_bench_gather4(_ptr(x), int(n), _ptr(sink), int(grid), int(iters), _stream_ptr(stream)))


def sell_bench_fma64(sink, grid: int, iters: int, stream=None):
    _check(load().sell_bench_fma64(_ptr(sink), int(grid), int(iters), _stream_ptr(stream)))


# ------------------------------------------------------------------ allocator
_alloc_keep = None


def use_torch_allocator(enable: bool = True):
    """Route the library's device allocations through PyTorch's caching
    allocator (so its memory shows up in torch's accounting)."""
    global _alloc_keep
    lib = load()
    if not enable:
        _check(lib.sell_set_allocator(ALLOC_FN(), FREE_FN(), None))
        _alloc_keep = None
        return
    import torch

    def _alloc(nbytes, ctx, stream):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      stream or 0)
        except Exception:
            return None

    def _free(ptr, ctx, stream):
        if ptr:
            torch.cuda.caching_allocator_delete(ptr)

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    _check(lib.sell_set_allocator(a, f, None))
    _alloc_keep = (a, f)


# ------------------------------------------------------------------ serving
def sell_server_create(mats, budget_bytes: int, max_batch: int = 64, streams: int = 3, size_ratio: int = 0,
                       max_batch_work: int = 0) -> int:
    arr = (_P * len(mats))(*[m.handle.value for m in mats])
    o = sell_server_opts(int(budget_bytes), int(max_batch), int(streams), int(size_ratio), 0, int(max_batch_work))
    out = _P()
    _check(load().sell_server_create(arr, len(mats), ctypes.byref(o), ctypes.byref(out)))
    return out.value


def sell_server_submit(srv: int, mid: int, X_ptr: int, k: int, Y_ptr: int | None, flags: int = 0) -> int:
    rid = ctypes.c_uint64()
    _check(load().sell_server_submit(_P(srv), int(mid), _P(X_ptr), int(k), _P(Y_ptr or 0), int(flags),
                                     ctypes.byref(rid)))
    return rid.value


def sell_server_wait(srv: int, rid: int, timeout_s: float = 60.0) -> sell_request_info:
    info = sell_request_info()
    _check(load().sell_server_wait(_P(srv), ctypes.c_uint64(rid), float(timeout_s), ctypes.byref(info)))
    return info


def sell_server_next(srv: int, timeout_s: float = 60.0):
    """(id, info) of the next completed request, in completion order."""
    rid = ctypes.c_uint64()
    info = sell_request_info()
    _check(load().sell_server_next(_P(srv), float(timeout_s), ctypes.byref(rid), ctypes.byref(info)))
    return rid.value, info


def sell_server_result(srv: int, rid: int) -> int:
    out = _P()
    _check(load().sell_server_result(_P(srv), ctypes.c_uint64(rid), ctypes.byref(out)))
    return out.value


def sell_server_release(srv: int, rid: int):
    _check(load().sell_server_release(_P(srv), ctypes.c_uint64(rid)))


def sell_server_stats(srv: int) -> dict:
    st = sell_server_stats_t()
    _check(load().sell_server_stats(_P(srv), ctypes.byref(st)))
    return {name: getattr(st, name) for name, _ in st._fields_}


def sell_server_destroy(srv: int):
    _check(load().sell_server_destroy(_P(srv)))
