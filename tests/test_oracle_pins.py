"""Pins for the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value comes from
exact rational arithmetic, a closed form of the paper, a textbook definition
written independently (ELLPACK, a dense product), or an invariant.
"""
import math
import struct
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1307_6209_gb300 import synth

U64 = 2.0 ** -53


def gamma(n, u=U64):
    return n * u / (1 - n * u)


# ----------------------------------------------------------------- Listing "crs"
@pytest.mark.parametrize("seed", range(6))
def test_csr_spmv_within_rounding_of_exact_rational(seed):
    """Listing "crs": the binary64 result is within gamma_n * sum|a x| of the
    exact rational value of sum_j a_ij x_j (recursive summation bound)."""
    A = synth.random_csr(11, 9, density=0.45, seed=seed, empty_rows=0.2)
    x = synth.vector(A.ncols, seed=100 + seed)
    y = oracle.csr_spmv(A, x)
    for i in range(A.nrows):
        lo, hi = A.rpt[i], A.rpt[i + 1]
        exact = sum((Fraction(float(A.val[j])) * Fraction(float(x[A.col[j]])) for j in range(lo, hi)),
                    Fraction(0))
        scale = sum(abs(float(A.val[j]) * float(x[A.col[j]])) for j in range(lo, hi))
        assert abs(Fraction(float(y[i])) - exact) <= Fraction(gamma(hi - lo + 1) * scale)
        if hi == lo:
            assert y[i] == 0.0 and math.copysign(1.0, y[i]) == 1.0


def test_csr_spmv_integer_matrix_is_exact():
    """Small integers: every product and partial sum is exact in binary64."""
    rng = np.random.default_rng(3)
    d = rng.integers(-5, 6, (40, 33)).astype(np.float64)
    d[rng.random(d.shape) < 0.6] = 0.0
    A = synth.from_dense(d)
    x = rng.integers(-7, 8, 33).astype(np.float64)
    y = oracle.csr_spmv(A, x)
    ref = [sum(int(d[i, j]) * int(x[j]) for j in range(33)) for i in range(40)]
    assert y.tolist() == [float(v) for v in ref]


@pytest.mark.parametrize("n,m", [(1, 1), (7, 64), (64, 64), (33, 5)])
def test_csr_spmv_dense_brute_force(n, m):
    """Dense brute force (numpy matmul on the densified matrix)."""
    A = synth.random_csr(n, m, density=0.3, seed=n * 100 + m)
    x = synth.vector(m, seed=7)
    d = A.to_dense()
    ref = d @ x
    scale = np.abs(d) @ np.abs(x)
    y = oracle.csr_spmv(A, x)
    assert np.all(np.abs(y - ref) <= 2 * gamma(m + 1) * scale + 1e-300)


def test_laplace_row_sums_with_unit_x():
    """5-point Laplacian, x = 1: interior rows sum to 0, edge rows to 1, corners to 2."""
    A = synth.laplace2d(64)
    y = oracle.csr_spmv(A, np.ones(A.ncols))
    g = y.reshape(64, 64)
    expect = np.zeros((64, 64))
    expect[0, :] += 1
    expect[-1, :] += 1
    expect[:, 0] += 1
    expect[:, -1] += 1
    assert np.array_equal(g, expect)


def test_csr_accumulate_starts_from_y():
    """Listing "crs" accumulates into y: with integer data y0 + A x is exact."""
    A = synth.laplace2d(8)
    x = np.arange(A.ncols, dtype=np.float64)
    y0 = np.arange(A.nrows, dtype=np.float64) * 3
    y = oracle.csr_spmv(A, x, y0=y0, accumulate=True)
    assert np.array_equal(y, y0 + A.to_dense() @ x)


def test_csr_threads_do_not_change_result():
    A = synth.lognormal(5000, seed=2)
    x = synth.vector(A.ncols, seed=2)
    y1 = oracle.csr_spmv(A, x, nthreads=1)
    y4 = oracle.csr_spmv(A, x, nthreads=4, guided=True)
    assert np.array_equal(y1, y4)


def test_csr_rows_matches_full_product_and_absdot():
    A = synth.lognormal(3000, seed=5)
    x = synth.vector(A.ncols, seed=5)
    y = oracle.csr_spmv(A, x)
    rows = np.array([0, 17, 2999, 1500, 17])
    yr, ab = oracle.csr_spmv_rows(A, x, rows)
    assert np.array_equal(yr, y[rows])
    d = A.to_dense()
    assert np.allclose(ab, (np.abs(d) @ np.abs(x))[rows], rtol=1e-13)


def test_absdot_is_dense_abs_product():
    """sum_j |a_ij x_j| (the scale of every tolerance) against |A| |x| computed
    densely; with small integers both are exact."""
    rng = np.random.default_rng(13)
    d = rng.integers(-9, 10, (30, 21)).astype(np.float64)
    d[rng.random(d.shape) < 0.5] = 0.0
    A = synth.from_dense(d)
    x = rng.integers(-6, 7, 21).astype(np.float64)
    assert np.array_equal(oracle.csr_absdot(A, x), np.abs(d) @ np.abs(x))


def test_spmmv_columns_are_independent_spmv():
    A = synth.random_csr(50, 40, density=0.2, seed=9)
    X = synth.block(40, 5, seed=1)
    Y = oracle.csr_spmmv(A, X)
    for c in range(5):
        assert np.array_equal(Y[:, c], oracle.csr_spmv(A, X[:, c].copy()))


# -------------------------------------------------------- the format (Sec. 3.3-3.4)
def _ellpack(A, rows_padded):
    """Textbook ELLPACK (Sec. 3.3): all rows padded to the longest one, stored
    column-major, row count padded; padding has value 0 and column 0."""
    rl = A.row_lengths()
    w = int(rl.max(initial=0))
    V = np.zeros((rows_padded, w))
    J = np.zeros((rows_padded, w), np.int32)
    for i in range(A.nrows):
        V[i, :rl[i]] = A.val[A.rpt[i]:A.rpt[i + 1]]
        J[i, :rl[i]] = A.col[A.rpt[i]:A.rpt[i + 1]]
    return V.T.reshape(-1), J.T.reshape(-1), w


@pytest.mark.parametrize("seed", range(3))
def test_sell_1_1_is_crs(seed):
    """Sec. 3.3: SELL-1-1 is CRS -- val/col byte-identical, cs == rpt, cl == rowLen."""
    A = synth.random_csr(37, 29, density=0.25, seed=seed, empty_rows=0.2)
    F = oracle.sell_build(A, 1, 1)
    assert F["val"].tobytes() == A.val.tobytes()
    assert np.array_equal(F["col"], A.col)
    assert np.array_equal(F["cs"], A.rpt)
    assert np.array_equal(F["cl"], A.row_lengths())
    assert np.array_equal(F["perm"], np.arange(A.nrows))
    assert F["beta"] == 1.0


@pytest.mark.parametrize("extra", [0, 5])
def test_sell_N_1_is_ellpack(extra):
    """Sec. 3.3: SELL-N-1 is ELLPACK (one chunk, width = longest row)."""
    A = synth.random_csr(45, 30, density=0.2, seed=4, empty_rows=0.1)
    C = A.nrows + extra
    F = oracle.sell_build(A, C, 1)
    V, J, w = _ellpack(A, C)
    assert F["nchunks"] == 1 and F["cl"].tolist() == [w]
    assert F["cs"].tolist() == [0, C * w]
    assert F["val"].tobytes() == V.tobytes()
    assert np.array_equal(F["col"], J)


def _check_sorted_windows(rl, perm, sigma):
    N = rl.shape[0]
    assert np.array_equal(np.sort(perm), np.arange(N))
    for w0 in range(0, N, max(sigma, 1)):
        w1 = min(w0 + max(sigma, 1), N)
        p = perm[w0:w1]
        assert p.min() >= w0 and p.max() < w1, "rows left their window"
        lens = rl[p]
        if sigma > 1:
            assert np.all(lens[:-1] >= lens[1:]), "not descending"
            ties = lens[:-1] == lens[1:]
            assert np.all(p[:-1][ties] < p[1:][ties]), "ties not stable"
        else:
            assert np.array_equal(p, np.arange(w0, w1))


@pytest.mark.parametrize("sigma", [1, 2, 3, 8, 64, 100, 1000, 10 ** 9])
def test_sigma_sort_invariants(sigma):
    """Sec. 3.4: rows sorted by length, descending, within windows of sigma rows;
    equal lengths keep their order; sigma >= N is the global sort (pJDS)."""
    A = synth.lognormal(777, seed=11, cap=60)
    F = oracle.sell_build(A, 8, sigma)
    _check_sorted_windows(A.row_lengths(), F["perm"], sigma)


def test_laplace_beta_closed_form():
    """Eq. "beta" for the 64x64 5-point Laplacian, SELL-32-1, derived by hand:
    chunks are half grid rows; the 4 chunks of the first and last grid rows have
    width 4 (edge rows), the other 124 chunks width 5.  Nnz = 5*4096 - 4*64."""
    A = synth.laplace2d(64)
    F = oracle.sell_build(A, 32, 1)
    stored = 32 * (4 * 4 + 124 * 5)
    nnz = 5 * 4096 - 4 * 64
    assert F["stored"] == stored and A.nnz == nnz
    assert F["beta"] == nnz / stored
    assert sorted(set(F["cl"].tolist())) == [4, 5]


@pytest.mark.parametrize("N,C", [(64, 4), (96, 8), (256, 16)])
def test_beta_worst_closed_form(N, C):
    """Eq. "betaworst": one full row and C-1 single-entry rows per chunk gives
    beta = (N + C - 1) / (C N) at sigma = 1."""
    A = synth.beta_worst(N, C)
    F = oracle.sell_build(A, C, 1)
    assert F["beta"] == pytest.approx((N + C - 1) / (C * N), rel=1e-15)


@pytest.mark.parametrize("N,C", [(64, 4), (128, 8), (256, 16)])
def test_beta_worst_sigma_c_squared_is_one(N, C):
    """Sec. 3.4: for the worst-case matrix sigma = C^2 gives beta = 1 (one chunk
    of full rows and C-1 chunks of length one per window)."""
    A = synth.beta_worst(N, C)
    F = oracle.sell_build(A, C, C * C)
    assert F["beta"] == 1.0
    assert F["cl"].tolist() == ([N] + [1] * (C - 1)) * (N // (C * C))


def test_constant_length_within_chunks_gives_beta_one():
    """Sec. 3.4: constant row length inside each chunk gives beta = 1."""
    rng = np.random.default_rng(1)
    C = 8
    lens = np.repeat(rng.integers(0, 20, 30), C)
    d = np.zeros((lens.shape[0], 25))
    for i, L in enumerate(lens):
        d[i, :L] = rng.uniform(0.5, 1.5, L)
    A = synth.from_dense(d)
    assert oracle.sell_build(A, C, 1)["beta"] == 1.0


@pytest.mark.parametrize("C,sigma", [(8, 2), (8, 4), (8, 8), (32, 16)])
def test_sigma_dividing_c_leaves_beta_unchanged(C, sigma):
    """Sec. 3.4: a sorting scope that divides C does not change beta."""
    A = synth.lognormal(1000, seed=3, cap=80)
    assert oracle.sell_build(A, C, sigma)["stored"] == oracle.sell_build(A, C, 1)["stored"]


def test_global_sort_minimises_storage():
    """sigma >= N (pJDS): after a global descending sort each chunk's width is
    its first row, so stored = C * sum of every C-th sorted length, the least
    storage over all row orders; every smaller scope stores at least as much."""
    A = synth.lognormal(4001, seed=8)  # N not a multiple of C: a partial last chunk
    C = 32
    srt = np.sort(A.row_lengths())[::-1]
    FN = oracle.sell_build(A, C, A.nrows)
    assert FN["stored"] == C * int(srt[::C].sum())
    for sigma in (1, 32, 256, 1024):
        assert oracle.sell_build(A, C, sigma)["stored"] >= FN["stored"]


def test_format_layout_by_definition():
    """Step 5 checked entry by entry: element j of sorted row r = c*C + l sits at
    cs[c] + j*C + l; everything else is zero padding with column 0."""
    A = synth.random_csr(23, 17, density=0.3, seed=12, empty_rows=0.2)
    C, sigma = 4, 8
    F = oracle.sell_build(A, C, sigma)
    seen = np.zeros(F["stored"], bool)
    for r in range(A.nrows):
        old = F["perm"][r]
        c, l = divmod(r, C)
        for j in range(A.rpt[old + 1] - A.rpt[old]):
            pos = F["cs"][c] + j * C + l
            assert F["val"][pos] == A.val[A.rpt[old] + j]
            assert F["col"][pos] == A.col[A.rpt[old] + j]
            seen[pos] = True
        assert F["srl"][r] == A.rpt[old + 1] - A.rpt[old]
    assert np.all(F["val"][~seen] == 0.0) and np.all(F["col"][~seen] == 0)
    assert np.all(F["srl"][A.nrows:] == 0)
    assert np.array_equal(np.diff(F["cs"]) // C, F["cl"])


def test_permuted_columns_are_symmetric_permutation():
    """Sec. 3.4 (column indices permuted with the rows): stored columns are
    invperm[col], i.e. the matrix P A P^T."""
    A = synth.lognormal(300, seed=4, cap=40)
    F = oracle.sell_build(A, 8, 64, permute_cols=True)
    G = oracle.sell_build(A, 8, 64, permute_cols=False)
    inv = np.empty_like(F["perm"])
    inv[F["perm"]] = np.arange(A.nrows)
    pad = G["val"] == 0
    assert np.array_equal(F["col"][~pad], inv[G["col"][~pad]])


# ------------------------------------------------------------- Listing "sell"
@pytest.mark.parametrize("C,sigma", [(1, 1), (2, 1), (4, 4), (32, 1), (32, 256), (64, 4096),
                                     (128, 10 ** 9), (7, 5), (3, 1000)])
def test_sell_spmv_bitwise_equals_crs(C, sigma):
    """The format keeps each row's summation order, and padding adds 0*x[0] = +-0
    to a sum that is never -0, so Listing "sell" equals Listing "crs" bitwise
    for finite x, for every (C, sigma)."""
    A = synth.lognormal(2100, seed=C + sigma % 97, cap=300)
    x = synth.vector(A.ncols, seed=1)
    y = oracle.csr_spmv(A, x)
    F = oracle.sell_build(A, C, sigma)
    assert np.array_equal(oracle.sell_spmv(F, x), y)
    y0 = synth.vector(A.nrows, seed=2)
    assert np.array_equal(oracle.sell_spmv(F, x, y0=y0, accumulate=True),
                          oracle.csr_spmv(A, x, y0=y0, accumulate=True))


def test_sell_spmv_permuted_space():
    """In sorted (permuted) space: y'[r] = y[perm[r]] for x'[r] = x[perm[r]]."""
    A = synth.lognormal(999, seed=6, cap=50)
    x = synth.vector(A.ncols, seed=3)
    F = oracle.sell_build(A, 16, 128, permute_cols=True)
    yp = oracle.sell_spmv(F, x[F["perm"]])
    assert np.array_equal(yp, oracle.csr_spmv(A, x)[F["perm"]])


def test_empty_and_degenerate():
    A = synth.CSR(0, 0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    F = oracle.sell_build(A, 32, 1)
    assert F["nchunks"] == 0 and F["stored"] == 0
    B = synth.CSR(5, 5, np.zeros(6, np.int64), np.zeros(0, np.int32), np.zeros(0))
    F = oracle.sell_build(B, 32, 4)
    assert F["stored"] == 0 and F["nchunks"] == 1
    assert np.array_equal(oracle.sell_spmv(F, np.ones(5)), np.zeros(5))


# ------------------------------------------------------------------- Eq. "cv"
def test_zeta_closed_forms():
    assert oracle.zeta(np.full(100, 7, np.int32)) == 0.0
    a, b = 3, 11
    rl = np.array([a, b] * 50, np.int32)
    assert oracle.zeta(rl) == pytest.approx(abs(a - b) / (a + b), rel=1e-14)


# ------------------------------------------------------------- value rounding
def _f32_bits(v):
    return struct.unpack("<I", struct.pack("<f", v))[0]


def test_round_f32_equals_ieee_cast():
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-40, 40, 10000),
                        [0.0, -0.0, 2.0 ** -149, 2.0 ** -150, 3 * 2.0 ** -151, 1e39, -1e39,
                         np.inf, -np.inf, 3.4028235677973366e38, 3.4028235677973362e38]])
    r = oracle.round_values(a, oracle.F32)
    with np.errstate(over="ignore"):
        ref = a.astype(np.float32)
    assert r.tobytes() == ref.tobytes()


@pytest.mark.parametrize("value,bits", [
    (1.0, 0x3F80),
    (1.0 + 2 ** -8, 0x3F80),                 # tie -> even (down)
    (1.0 + 3 * 2 ** -8, 0x3F82),             # tie -> even (up)
    (1.0 + 2 ** -8 + 2 ** -30, 0x3F81),      # just above the tie
    (1.0 + 2 ** -8 + 2 ** -40, 0x3F81),      # binary32-first would round down
    (-2.5, 0xC020),
    ((2 - 2 ** -7) * 2.0 ** 127, 0x7F7F),    # largest finite
    (2.0 ** 128 - 2.0 ** 119, 0x7F80),       # overflow midpoint -> inf
    (2.0 ** 128 - 2.0 ** 119 - 2.0 ** 100, 0x7F7F),
    (2.0 ** -133, 0x0001),                   # smallest subnormal
    (2.0 ** -134, 0x0000),                   # half of it: tie -> even (zero)
    (1.5 * 2.0 ** -134, 0x0001),
    (2.0 ** -126, 0x0080),                   # smallest normal
    (-0.0, 0x8000),
    (float("inf"), 0x7F80),
])
def test_round_bf16_hand_derived(value, bits):
    """bfloat16 = 1 sign, 8 exponent, 7 fraction bits; one rounding, ties to even."""
    r = oracle.round_values(np.array([value]), oracle.BF16)
    assert int(r[0]) == bits


def test_round_bf16_is_nearest():
    """Brute force: the rounded value is the nearest of its two bf16 neighbours."""
    rng = np.random.default_rng(5)
    a = rng.standard_normal(20000) * 10.0 ** rng.integers(-30, 30, 20000)
    # and the subnormal range, 2^-133 (smallest subnormal) up to 2^-126
    a = np.concatenate([a, rng.uniform(-1, 1, 5000) * 2.0 ** rng.integers(-135, -125, 5000)])
    r = oracle.round_values(a, oracle.BF16).astype(np.int64)
    v = oracle.bf16_to_f64(r.astype(np.uint16))
    up = oracle.bf16_to_f64(((r & 0x7FFF) + 1 | (r & 0x8000)).astype(np.uint16))
    dn = oracle.bf16_to_f64((np.maximum((r & 0x7FFF) - 1, 0) | (r & 0x8000)).astype(np.uint16))
    err = np.abs(v - a)
    assert np.all(err <= np.abs(up - a)) and np.all(err <= np.abs(dn - a))
