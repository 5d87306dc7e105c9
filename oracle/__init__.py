"""CPU oracle for SELL-C-sigma (arXiv:1307.6209) -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct binary64 implementations of what the CUDA
library computes.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with ``paper_1307_6209_gb300`` and imports nothing from it.

The arithmetic lives in ``sell_oracle.c`` (compiled with gcc, no FMA
contraction); this module only marshals numpy arrays.  Matrices are passed as
any object with ``nrows, ncols, rpt (int64[N+1]), col (int32[nnz]),
val (float64[nnz])`` attributes.

Function -> paper passage:
  csr_spmv, csr_spmv_rows, csr_spmmv : Sec. 3.1, Listing "crs"
  sell_build                         : Sec. 3.3-3.4, Eqs. "nc", "max"; padding
                                       convention of Sec. 4
  sell_spmv                          : Sec. 3.3, Listing "sell" (general C)
  beta                               : Sec. 3.4, Eq. "beta"
  zeta                               : Sec. 5, Eq. "cv"
  round_values                       : reduced-precision storage (not in the
                                       paper; single round-to-nearest-even)
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sell_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

F32, BF16 = 1, 2


def compile_library(src: str, out: str) -> str:
    """Compile a C oracle source into a shared library (OpenMP if available)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", src, "-o", out + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(out + ".tmp", out)
    return out


def build(force: bool = False) -> str:
    """Compile sell_oracle.c with gcc (OpenMP if available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    return compile_library(_SRC, _LIB)


def _bind(path: str):
    lib = ctypes.CDLL(path)
    p = ctypes.c_void_p
    i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    sig = {
        "orc_csr_spmv": (None, [i64, p, p, p, p, p, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "orc_csr_spmv_rows": (None, [p, p, p, p, p, i64, p, p]),
        "orc_csr_spmmv": (None, [i64, p, p, p, i32, p, i64, p, i64, ctypes.c_int]),
        "orc_csr_absdot": (None, [i64, p, p, p, p, p]),
        "orc_sell_plan": (ctypes.c_int, [i64, p, i32, i64, p, p, p, p]),
        "orc_sell_fill": (ctypes.c_int, [i64, i64, p, p, p, i32, p, p, p, p, ctypes.c_int, p, p, p]),
        "orc_sell_spmv": (None, [i64, i32, p, p, p, p, p, p, p, ctypes.c_int, ctypes.c_int]),
        "orc_beta": (f64, [i64, i64, i32, p]),
        "orc_zeta": (f64, [i64, p]),
        "orc_round": (None, [i64, p, ctypes.c_int, p]),
        "orc_bf16_to_f64": (None, [i64, p, p]),
        "orc_max_threads": (ctypes.c_int, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
        return _lib


@contextlib.contextmanager
def substituted_library(path: str):
    """Run this module's functions on another build of the C source for the
    duration of the block.  Used only by the mutation tests, which plant one
    mistake in a copy of sell_oracle.c and check that a pin catches it."""
    global _lib
    lib = _bind(path)
    with _lock:
        saved, _lib = _lib, lib
    try:
        yield
    finally:
        with _lock:
            _lib = saved


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _csr(A):
    return (int(A.nrows), int(A.ncols), _c(A.rpt, np.int64), _c(A.col, np.int32),
            _c(A.val, np.float64))


def max_threads() -> int:
    return int(_load().orc_max_threads())


# --------------------------------------------------------------------------- CRS
def csr_spmv(A, x, y0=None, accumulate=False, nthreads=0, guided=False):
    """Listing "crs": y = A x (or y = y0 + A x), binary64, CRS summation order."""
    lib = _load()
    n, m, rpt, col, val = _csr(A)
    x = _c(x, np.float64)
    assert x.shape[0] >= m
    y = np.zeros(n, np.float64) if y0 is None else _c(y0, np.float64).copy()
    lib.orc_csr_spmv(n, _ptr(rpt), _ptr(col), _ptr(val), _ptr(x), _ptr(y),
                     1 if accumulate else 0, int(nthreads), 1 if guided else 0)
    return y


def csr_spmv_rows(A, x, rows):
    """Listing "crs" for selected rows; returns (y_rows, sum_j |a_ij x_j|)."""
    lib = _load()
    _, _, rpt, col, val = _csr(A)
    x = _c(x, np.float64)
    rows = _c(rows, np.int64)
    out = np.empty(rows.shape[0], np.float64)
    ab = np.empty(rows.shape[0], np.float64)
    lib.orc_csr_spmv_rows(_ptr(rpt), _ptr(col), _ptr(val), _ptr(x), _ptr(rows),
                          rows.shape[0], _ptr(out), _ptr(ab))
    return out, ab


def csr_spmmv(A, X, Y0=None, accumulate=False):
    """Y[:, c] = A X[:, c] (+ Y0[:, c]) for every column c of the row-major X."""
    lib = _load()
    n, m, rpt, col, val = _csr(A)
    X = _c(X, np.float64)
    k = X.shape[1]
    Y = np.zeros((n, k), np.float64) if Y0 is None else _c(Y0, np.float64).copy()
    lib.orc_csr_spmmv(n, _ptr(rpt), _ptr(col), _ptr(val), k, _ptr(X), X.shape[1],
                      _ptr(Y), Y.shape[1], 1 if accumulate else 0)
    return Y


def csr_absdot(A, x):
    """Row-wise sum_j |a_ij x_j| in binary64."""
    lib = _load()
    n, _, rpt, col, val = _csr(A)
    x = _c(x, np.float64)
    out = np.empty(n, np.float64)
    lib.orc_csr_absdot(n, _ptr(rpt), _ptr(col), _ptr(val), _ptr(x), _ptr(out))
    return out


# --------------------------------------------------------------------- SELL-C-sigma
def sell_build(A, C, sigma, permute_cols=False):
    """Steps 1-5 of the format (Sec. 3.3-3.4).  Returns a dict with rl (original
    order), perm (sorted -> original), cl, cs, val (binary64), col, srl (length
    of each sorted row, Nc*C entries), nchunks, stored, beta, zeta."""
    lib = _load()
    n, m, rpt, col, val = _csr(A)
    C = int(C)
    sigma = int(sigma)
    nc = (n + C - 1) // C
    rl = np.empty(n, np.int32)
    perm = np.empty(n, np.int32)
    cl = np.empty(nc, np.int32)
    cs = np.empty(nc + 1, np.int64)
    rc = lib.orc_sell_plan(n, _ptr(rpt), C, sigma, _ptr(rl), _ptr(perm), _ptr(cl), _ptr(cs))
    if rc != 0:
        raise ValueError(f"orc_sell_plan failed ({rc})")
    stored = int(cs[nc])
    sval = np.empty(stored, np.float64)
    scol = np.empty(stored, np.int32)
    srl = np.empty(nc * C, np.int32)
    rc = lib.orc_sell_fill(n, m, _ptr(rpt), _ptr(col), _ptr(val), C, _ptr(rl), _ptr(perm),
                           _ptr(cl), _ptr(cs), 1 if permute_cols else 0, _ptr(sval),
                           _ptr(scol), _ptr(srl))
    if rc != 0:
        raise ValueError(f"orc_sell_fill failed ({rc})")
    nnz = int(rpt[n]) if n > 0 else 0
    return {
        "nrows": n, "ncols": m, "nnz": nnz, "C": C, "sigma": sigma,
        "rl": rl, "perm": perm, "cl": cl, "cs": cs, "val": sval, "col": scol, "srl": srl,
        "nchunks": nc, "stored": stored,
        "beta": float(lib.orc_beta(nnz, nc, C, _ptr(cl))),
        "zeta": float(lib.orc_zeta(n, _ptr(rl))),
        "permute_cols": bool(permute_cols),
    }


def sell_spmv(F, x, y0=None, accumulate=False):
    """Listing "sell" for general C over the oracle's own format dict F."""
    lib = _load()
    n = F["nrows"]
    x = _c(x, np.float64)
    y = np.zeros(n, np.float64) if y0 is None else _c(y0, np.float64).copy()
    lib.orc_sell_spmv(n, F["C"], _ptr(F["perm"]), _ptr(F["cl"]), _ptr(F["cs"]),
                      _ptr(F["val"]), _ptr(F["col"]), _ptr(x), _ptr(y),
                      1 if accumulate else 0, 1 if F["permute_cols"] else 0)
    return y


def beta(nnz, C, cl):
    cl = _c(cl, np.int32)
    return float(_load().orc_beta(int(nnz), cl.shape[0], int(C), _ptr(cl)))


def zeta(rl):
    rl = _c(rl, np.int32)
    return float(_load().orc_zeta(rl.shape[0], _ptr(rl)))


# ------------------------------------------------------------- reduced precision
def round_values(a, to):
    """Round binary64 values once, to nearest even: to=F32 -> float32 array,
    to=BF16 -> uint16 array of bfloat16 bit patterns."""
    lib = _load()
    a = _c(a, np.float64)
    out = np.empty(a.shape[0], np.float32 if to == F32 else np.uint16)
    lib.orc_round(a.shape[0], _ptr(a), int(to), _ptr(out))
    return out


def bf16_to_f64(bits):
    lib = _load()
    bits = _c(bits, np.uint16)
    out = np.empty(bits.shape[0], np.float64)
    lib.orc_bf16_to_f64(bits.shape[0], _ptr(bits), _ptr(out))
    return out
