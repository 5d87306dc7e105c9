"""The paper's performance model (Sec. 4) and the byte counts the benchmark
reports against it.

Code balance (bytes per flop) of the binary64 SpMV with four-byte indices:
  CRS   : B = 6 + 4 alpha + 8 / Nnzr                      (Eq. "crsbalance")
  SELL  : B = 6 / beta + 4 alpha + 8 / Nnzr               (Eq. "sellbalance")
Roofline: P = b / B (Eq. "roof_general"); with alpha = 1/Nnzc (Eq. "roof_alpha")
and Nnzr >> 12 the bound becomes P = b beta / 6 (Eq. "best_veccache").
alpha from a measured volume V (memory-bound runs only, Eq. "eq:sellalpha"):
  alpha = ( V / (2 Nnz) - 6 / beta - 8 / Nnzr ) / 4.
The 8/Nnzr term is v_LHS = 16 B per row (y read and written, as in the
paper's accumulating listings); this library's default y = A x writes y only
(8 B per row), which ``algorithmic_bytes`` counts.
"""
from __future__ import annotations


def balance_crs(alpha: float, nnzr: float) -> float:
    return 6.0 + 4.0 * alpha + 8.0 / nnzr


def balance_sell(alpha: float, beta: float, nnzr: float) -> float:
    return 6.0 / beta + 4.0 * alpha + 8.0 / nnzr


def roofline(b_gbs: float, balance: float) -> float:
    """GF/s bound for bandwidth b (GB/s) and code balance (bytes/flop)."""
    return b_gbs / balance


def best_bound(b_gbs: float, beta: float = 1.0) -> float:
    """Eq. "best_veccache": P = b beta / 6."""
    return b_gbs * beta / 6.0


def alpha_from_volume(v_bytes: float, nnz: int, beta: float, nnzr: float) -> float:
    return 0.25 * (v_bytes / (2.0 * nnz) - 6.0 / beta - 8.0 / nnzr)


def algorithmic_bytes(nrows: int, ncols: int, nnz: int, nchunks: int, C: int, value_bytes: int,
                      x_bytes: int, has_perm: bool, k: int = 1, accumulate: bool = False) -> int:
    """Least bytes one SELL-C-sigma product must move with the ELLR-T skip:
    every stored nonzero once (value + 4-byte column), x once (alpha =
    1/Nnzc), y written (and read when accumulating), the sorted row lengths
    (4 B per padded row), the permutation (4 B per row when sigma > 1) and
    the chunk offsets (8 B per chunk)."""
    b = (value_bytes + 4) * nnz
    b += x_bytes * ncols * k
    b += x_bytes * nrows * k * (2 if accumulate else 1)
    b += 4 * nchunks * C
    b += 4 * nrows if has_perm else 0
    b += 8 * (nchunks + 1)
    return int(b)


def paper_model_bytes(nnz: int, beta: float, nrows: int, ncols: int, value_bytes: int = 8,
                      x_bytes: int = 8) -> float:
    """Bytes of the paper's model with alpha = 1/Nnzc (Eqs. "sellbalance",
    "roof_alpha"): (value + index)/beta per nonzero, x once, y read + write."""
    return (value_bytes + 4) * nnz / beta + x_bytes * ncols + 2 * x_bytes * nrows
