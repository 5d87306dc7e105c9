"""Property tests of the CPU oracle (hypothesis): random small CRS matrices and
random (C, sigma) against definitions written out here, independently.

* Listing "sell" over the format equals Listing "crs" bit for bit (the format
  keeps each row's summation order; padding adds signed zeros to a sum that is
  never -0).
* The format arrays satisfy their definition entry by entry (Sec. 3.3-3.4).
* The sort is descending and stable inside each sigma-window.
* Eq. "beta" is nnz over the stored elements, and 0 < beta <= 1.
* A CRS product of small integers equals the exact integer product.
* Rounding to binary32 is the IEEE conversion; to bfloat16 the nearest value.
"""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle  # noqa: E402
from paper_1307_6209_gb300 import synth  # noqa: E402

SETTINGS = settings(max_examples=150, deadline=None, derandomize=True)


@st.composite
def csr_matrices(draw, max_n=40, max_m=40, integer=False):
    n = draw(st.integers(0, max_n))
    m = draw(st.integers(1, max_m))
    lens = draw(st.lists(st.integers(0, m), min_size=n, max_size=n))
    rng = np.random.default_rng(draw(st.integers(0, 2 ** 32 - 1)))
    cols = [np.sort(rng.choice(m, size=k, replace=False)) for k in lens]
    col = np.concatenate(cols).astype(np.int32) if n else np.zeros(0, np.int32)
    if integer:
        val = rng.integers(-6, 7, col.shape[0]).astype(np.float64)
    else:
        val = rng.standard_normal(col.shape[0]) * 10.0 ** rng.integers(-3, 4, col.shape[0])
    rpt = np.zeros(n + 1, np.int64)
    np.cumsum(lens, out=rpt[1:])
    return synth.CSR(n, m, rpt, col, val)


formats = st.tuples(st.integers(1, 70), st.one_of(st.integers(1, 100), st.just(10 ** 9)))


@SETTINGS
@given(csr_matrices(), formats, st.booleans())
def test_sell_spmv_equals_crs_bitwise(A, fmt, accumulate):
    C, sigma = fmt
    rng = np.random.default_rng(A.nnz + C)
    x = rng.uniform(-1, 1, A.ncols)
    y0 = rng.uniform(-1, 1, A.nrows) if accumulate else None
    F = oracle.sell_build(A, C, sigma)
    ref = oracle.csr_spmv(A, x, y0=y0, accumulate=accumulate)
    got = oracle.sell_spmv(F, x, y0=y0, accumulate=accumulate)
    assert got.tobytes() == ref.tobytes()


@SETTINGS
@given(csr_matrices(), formats)
def test_format_arrays_by_definition(A, fmt):
    C, sigma = fmt
    F = oracle.sell_build(A, C, sigma)
    N = A.nrows
    rl = np.diff(A.rpt)
    nc = -(-N // C)
    assert F["nchunks"] == nc and F["cs"].shape[0] == nc + 1
    perm = F["perm"]
    assert np.array_equal(np.sort(perm), np.arange(N))
    # sorted row lengths, padded rows empty
    srl = np.zeros(nc * C, np.int64)
    srl[:N] = rl[perm]
    assert np.array_equal(F["srl"], srl)
    # Eq. "max" and the offsets
    cl = srl.reshape(nc, C).max(axis=1) if nc else np.zeros(0, np.int64)
    assert np.array_equal(F["cl"], cl)
    assert np.array_equal(F["cs"], np.concatenate([[0], np.cumsum(C * cl)]))
    # entry j of sorted row r = c*C + l at cs[c] + j*C + l; the rest is zero padding
    val = np.zeros(int(F["cs"][-1]))
    col = np.zeros(int(F["cs"][-1]), np.int32)
    for r in range(N):
        c, l = divmod(r, C)
        lo = A.rpt[perm[r]]
        for j in range(rl[perm[r]]):
            val[F["cs"][c] + j * C + l] = A.val[lo + j]
            col[F["cs"][c] + j * C + l] = A.col[lo + j]
    assert F["val"].tobytes() == val.tobytes() and np.array_equal(F["col"], col)
    # Eq. "beta"
    stored = int(F["cs"][-1])
    assert F["stored"] == stored >= A.nnz
    assert F["beta"] == (A.nnz / stored if stored else 1.0)


@SETTINGS
@given(csr_matrices(max_n=60), st.integers(1, 80))
def test_sort_descending_stable_in_windows(A, sigma):
    F = oracle.sell_build(A, 4, sigma)
    rl = np.diff(A.rpt)
    for w0 in range(0, A.nrows, sigma):
        w1 = min(w0 + sigma, A.nrows)
        p = F["perm"][w0:w1]
        assert p.min() >= w0 and p.max() < w1
        # the stable descending order is unique: longest first, ties by row
        expect = sorted(range(w0, w1), key=lambda i: (-rl[i], i)) if sigma > 1 else list(range(w0, w1))
        assert p.tolist() == expect


@SETTINGS
@given(csr_matrices(integer=True))
def test_crs_integer_product_is_exact(A):
    rng = np.random.default_rng(A.nnz)
    x = rng.integers(-9, 10, A.ncols).astype(np.float64)
    y = oracle.csr_spmv(A, x)
    d = A.to_dense().astype(np.int64)
    assert y.tolist() == [float(v) for v in d @ x.astype(np.int64)]
    X = rng.integers(-9, 10, (A.ncols, 3)).astype(np.float64)
    Y = oracle.csr_spmmv(A, X)
    assert np.array_equal(Y, (d @ X.astype(np.int64)).astype(np.float64))


finite = st.floats(allow_nan=False, allow_infinity=False, width=64)


@SETTINGS
@given(st.lists(finite, min_size=1, max_size=50))
def test_round_f32_is_ieee_conversion(vals):
    a = np.array(vals)
    with np.errstate(over="ignore"):
        ref = a.astype(np.float32)
    assert oracle.round_values(a, oracle.F32).tobytes() == ref.tobytes()


@SETTINGS
@given(st.lists(st.floats(min_value=-3e38, max_value=3e38, allow_nan=False), min_size=1, max_size=50))
def test_round_bf16_is_nearest(vals):
    a = np.array(vals)
    r = oracle.round_values(a, oracle.BF16).astype(np.int64)
    v = oracle.bf16_to_f64(r.astype(np.uint16))
    mag = r & 0x7FFF
    up = oracle.bf16_to_f64(((mag + 1) | (r & 0x8000)).astype(np.uint16))
    dn = oracle.bf16_to_f64((np.maximum(mag - 1, 0) | (r & 0x8000)).astype(np.uint16))
    err = np.abs(v - a)
    assert np.all(err <= np.abs(up - a)) and np.all(err <= np.abs(dn - a))
    # ties go to an even significand
    tie = (err == np.abs(up - a)) | (err == np.abs(dn - a))
    assert np.all((mag[tie & (err > 0)] & 1) == 0)
