"""Helpers shared by the GPU parity tests (imported only by tests)."""
import numpy as np

import oracle
from paper_1307_6209_gb300 import synth

U64 = 2.0 ** -53
U32 = 2.0 ** -24


def gamma(n, u):
    n = np.asarray(n, np.float64)
    return n * u / (1.0 - n * u)


def tol_f64(rl, scale):
    """Row-wise bound for a binary64 FMA chain against the binary64 oracle:
    both sides are within gamma_n * sum|a x| of the exact value, and the
    stated tolerance is 1e-12 of sum|a x| (or 2 gamma_n for rows beyond
    ~4500 entries, where 1e-12 is below the rounding bound)."""
    return np.maximum(1e-12, 2.0 * gamma(rl + 1, U64)) * scale + 1e-300


def tol_f32(rl, scale):
    """Binary32 FMA chain of n steps: |y - s| <= gamma_n(2^-24) sum|a x|."""
    return 1.01 * gamma(rl + 1, U32) * scale + 2.0 ** -140


def tol_dot2(rl, scale, ref):
    """Dot2 (Ogita-Rump-Oishi, Prop. 5.5): |res - s| <= u|s| + gamma_n^2 sum|a x|."""
    return 1.01 * (U32 * np.abs(ref) + gamma(rl + 1, U32) ** 2 * scale) + 2.0 ** -140


def parity_matrices():
    """(name, CSR) cases spanning several chunks, ragged tails and the
    degenerate shapes: empty rows, N not a multiple of C, N < C, nnz = 0, a
    single long row, the beta worst case."""
    return [
        ("laplace64", synth.laplace2d(64)),
        ("lognormal5k", synth.lognormal(5003, seed=1, cap=300)),
        ("random_empty_rows", synth.random_csr(777, 500, density=0.02, seed=2, empty_rows=0.3)),
        ("tiny_N_lt_C", synth.random_csr(13, 9, density=0.4, seed=3)),
        ("nnz0", synth.CSR(100, 50, np.zeros(101, np.int64), np.zeros(0, np.int32), np.zeros(0))),
        ("long_row", synth.long_row(3000, 2500, short_len=3, at=1234, seed=4)),
        ("beta_worst", synth.beta_worst(256, 16)),
        ("rect_wide", synth.random_csr(300, 2000, density=0.01, seed=5)),
        ("banded", synth.banded(4099, seed=6)),
    ]


def oracle_reference(A, x):
    """(y, sum|a x|, row lengths) from the oracle."""
    return oracle.csr_spmv(A, x), oracle.csr_absdot(A, x), A.row_lengths()
