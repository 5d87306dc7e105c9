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


def rounded_csr(A, store):
    """A with its values rounded once to the storage type (0 binary64,
    1 binary32, 2 bfloat16) by the oracle, as binary64: the matrix the kernel
    actually multiplies."""
    if store == 0:
        return A
    r = oracle.round_values(A.val, store)
    v = r.astype(np.float64) if store == 1 else oracle.bf16_to_f64(r)
    return synth.CSR(A.nrows, A.ncols, A.rpt, A.col, v)


def host_csr(A):
    """Host (numpy) copy of a CSR whose arrays may be CUDA tensors."""
    if isinstance(A.rpt, np.ndarray):
        return A
    return synth.CSR(A.nrows, A.ncols, A.rpt.cpu().numpy(), A.col.cpu().numpy(),
                     A.val.cpu().numpy().astype(np.float64))


def assert_oracle_parity(A, store, X, Y, flags=0, Y0=None, what=""):
    """Every column of a GPU result Y (nrows, or nrows x k) against the
    oracle's binary64 CRS product (Listing "crs") on the stored values, within
    the bound of the arithmetic the kernel ran: tol_f64 for binary64 storage,
    tol_f32 for binary32 chains, tol_dot2 for compensated rows (flags 0x2 on
    every row, 0x8 on rows of more than 64 entries).  flags 0x1 adds Y0."""
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    acc = bool(flags & 0x1)
    if X.ndim == 1:
        X, Y = X[:, None], Y[:, None]
        if Y0 is not None:
            Y0 = np.asarray(Y0)[:, None]
    if acc:
        Y0 = np.asarray(Y0, np.float64)
    Ar = rounded_csr(A, store)
    rl = A.row_lengths()
    n = rl + (1 if acc else 0)
    for c in range(X.shape[1]):
        x = X[:, c]
        ref = oracle.csr_spmv(Ar, x, y0=Y0[:, c] if acc else None, accumulate=acc)
        scale = oracle.csr_absdot(Ar, x) + (np.abs(Y0[:, c]) if acc else 0.0)
        if store == 0:
            tol = tol_f64(n, scale)
        elif flags & 0x2:
            tol = tol_dot2(n, scale, ref)
        elif flags & 0x8:
            tol = np.where(rl > 64, tol_dot2(n, scale, ref), tol_f32(n, scale))
        else:
            tol = tol_f32(n, scale)
        err = np.abs(Y[:, c] - ref)
        bad = np.nonzero(~(err <= tol))[0]
        assert bad.size == 0, (f"{what} column {c}: {bad.size} rows outside the bound, first row {bad[0]}: "
                               f"got {Y[bad[0], c]!r}, oracle {ref[bad[0]]!r}, tol {tol[bad[0]]!r}")
