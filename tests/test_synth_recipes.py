"""The synthetic inputs follow the recipe they are documented with.

The paper's matrices (University of Florida collection) are not available, so
seeded synthetic matrices stand in for them.  These CPU tests check each
generator -- the numpy versions and the torch versions (run here on the CPU
device) that make the large inputs on the GPU -- against its stated recipe:
exact counts where the structure fixes them, and distribution checks against
values computed independently (the lognormal CDF) where it is random.
"""
import math

import numpy as np
import pytest

from paper_1307_6209_gb300 import synth


def _np(a):
    return a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a)


def _check_csr(A, *, square=True):
    rpt, col = _np(A.rpt), _np(A.col).astype(np.int64)
    assert rpt[0] == 0 and np.all(np.diff(rpt) >= 0) and rpt[-1] == col.shape[0]
    assert col.min(initial=0) >= 0 and col.max(initial=-1) < A.ncols
    if square:
        assert A.nrows == A.ncols
    # distinct and ascending inside every row
    rows = np.repeat(np.arange(A.nrows), np.diff(rpt))
    same_row = rows[1:] == rows[:-1]
    assert np.all(col[1:][same_row] > col[:-1][same_row])


# ------------------------------------------------------------------ stencils
@pytest.mark.parametrize("n", [1, 2, 5, 9])
def test_laplace2d_structure(n):
    A = synth.laplace2d(n)
    _check_csr(A)
    assert A.nnz == 5 * n * n - 4 * n
    d = A.to_dense()
    assert np.array_equal(d, d.T)
    assert np.all(np.diag(d) == 4.0)
    off = d - np.diag(np.diag(d))
    assert set(np.unique(off)) <= {0.0, -1.0}


@pytest.mark.parametrize("n", [1, 2, 3, 7])
def test_stencil27_structure(n):
    A = synth.stencil27(n)
    _check_csr(A)
    assert A.nnz == (3 * n - 2) ** 3  # 598^3 = 213,847,192 at n = 200
    d = A.to_dense()
    assert np.array_equal(d != 0, (d != 0).T)
    assert np.all(np.diag(d) == 26.0)
    # an interior row sums to 26 - 26 = 0
    if n >= 3:
        c = n // 2
        i = (c * n + c) * n + c
        assert d[i].sum() == 0.0 and (d[i] != 0).sum() == 27


def test_stencil27_perturbation_bounds():
    p = 0.1
    A = synth.stencil27(6, perturb=p, seed=3)
    B = synth.stencil27(6)
    assert np.array_equal(A.col, B.col) and np.array_equal(A.rpt, B.rpt)
    r = A.val / B.val
    assert np.all((r >= 1 - p) & (r <= 1 + p)) and np.std(r) > p / 4


def test_stencil27_row_prefix_equals_the_full_matrix():
    """The reference arm's row sample: the first r rows of the stencil,
    values included, are the prefix of the full matrix's arrays."""
    full = synth.stencil27(9, perturb=0.1, seed=3)
    for r in (0, 1, 80, 400, 729, 10 ** 6):
        P = synth.stencil27(9, perturb=0.1, seed=3, rows=r)
        m = min(r, full.nrows)
        assert P.nrows == m and P.ncols == full.ncols
        assert np.array_equal(P.rpt, full.rpt[:m + 1])
        assert np.array_equal(P.col, full.col[:full.rpt[m]])
        assert np.array_equal(P.val, full.val[:full.rpt[m]])


@pytest.mark.parametrize("n", [1, 4, 7])
def test_stencil27_device_matches_host_structure(n):
    A = synth.stencil27(n)
    D = synth.stencil27_device(n, perturb=0.0, device="cpu")
    assert np.array_equal(_np(D.rpt), A.rpt)
    assert np.array_equal(_np(D.col), A.col)
    assert np.array_equal(_np(D.val), A.val)
    P = synth.stencil27_device(n, perturb=0.1, seed=1, device="cpu")
    r = _np(P.val) / A.val
    assert np.all((r >= 0.9) & (r <= 1.1))


# ------------------------------------------------------------- lognormal rows
def _rounded_clamped_lognormal_pmf(mean, sigma_ln, cap):
    """P(clip(rint(X), 1, cap) = k) for X lognormal with E[X] = mean, from the
    normal CDF (rint rounds half to even, which has probability zero here)."""
    mu = math.log(mean) - 0.5 * sigma_ln ** 2

    def cdf(x):
        return 0.5 * (1.0 + math.erf((math.log(x) - mu) / (sigma_ln * math.sqrt(2.0))))

    p = np.empty(cap + 1)
    p[0] = 0.0
    p[1] = cdf(1.5)
    for k in range(2, cap):
        p[k] = cdf(k + 0.5) - cdf(k - 0.5)
    p[cap] = 1.0 - cdf(cap - 0.5)
    return p


@pytest.mark.parametrize("gen", ["numpy", "torch"])
def test_lognormal_row_length_distribution(gen):
    N, mean, s, cap = 400_000, 16.0, 1.2, 2000
    if gen == "numpy":
        rl = synth.lognormal_lengths(N, mean, s, cap, np.random.default_rng(7))
    else:
        import torch
        A = synth.lognormal_device(20_000, mean, s, cap, seed=7, device="cpu")
        _check_csr(A)
        # the lengths of the torch recipe, drawn the way lognormal_device draws them
        g = torch.Generator(device="cpu")
        g.manual_seed(7)
        z = torch.randn(20_000, generator=g, dtype=torch.float64)
        mu = math.log(mean) - 0.5 * s * s
        assert np.array_equal(np.diff(_np(A.rpt)),
                              np.clip(np.rint(np.exp(mu + s * z.numpy())), 1, cap).astype(np.int64))
        g.manual_seed(8)
        z = torch.randn(N, generator=g, dtype=torch.float64).numpy()
        rl = np.clip(np.rint(np.exp(mu + s * z)), 1, cap).astype(np.int64)
    pmf = _rounded_clamped_lognormal_pmf(mean, s, cap)
    k = np.arange(cap + 1)
    m, var = float((k * pmf).sum()), float((k * k * pmf).sum() - (k * pmf).sum() ** 2)
    assert rl.min() >= 1 and rl.max() <= cap
    assert abs(rl.mean() - m) < 5 * math.sqrt(var / N)
    assert abs(m - mean) < 0.05  # rounding and the clamp barely move the mean
    for j in (1, 2, 16):  # point masses, each within 5 standard errors
        f = float(np.mean(rl == j))
        assert abs(f - pmf[j]) < 5 * math.sqrt(pmf[j] * (1 - pmf[j]) / N)


def test_lognormal_matrix_recipe():
    A = synth.lognormal(30_000, seed=4)
    _check_csr(A)
    rl = A.row_lengths()
    assert np.array_equal(rl, synth.lognormal_lengths(30_000, rng=np.random.default_rng(4)))
    assert abs(A.val.mean()) < 0.01 and abs(A.val.std() - 1.0) < 0.01
    # columns uniform over [0, N): each tenth of the range holds about a tenth
    h = np.bincount(A.col.astype(np.int64) * 10 // A.ncols, minlength=10) / A.nnz
    assert np.all(np.abs(h - 0.1) < 0.005)


def test_lognormal_headline_size():
    """The benchmark's matrix: N = 2,000,000, seed 0."""
    A = synth.lognormal(2_000_000, seed=0)
    assert A.nnz == 32_058_194
    assert int(A.row_lengths().max()) <= 2000


def test_lognormal_cap_never_exceeds_n():
    A = synth.lognormal(50, seed=1, cap=2000)
    _check_csr(A)
    assert A.row_lengths().max() <= 50


# ------------------------------------------------------------------- banded
@pytest.mark.parametrize("gen", ["numpy", "torch"])
def test_banded_recipe(gen):
    N, bw, lo, hi = 5000, 64, 7, 30
    A = synth.banded(N, bw, lo, hi, seed=2) if gen == "numpy" else \
        synth.banded_device(N, bw, lo, hi, seed=2, device="cpu")
    _check_csr(A)
    rpt, col = _np(A.rpt), _np(A.col).astype(np.int64)
    rl = np.diff(rpt)
    rows = np.repeat(np.arange(N), rl)
    assert np.all(np.abs(col - rows) <= bw)
    inner = rl[bw:N - bw]
    assert inner.min() == lo and inner.max() == hi
    assert abs(inner.mean() - (lo + hi) / 2) < 0.5
    assert np.all(rl >= 1) and np.all(rl <= hi)


# ------------------------------------------------------------- special shapes
@pytest.mark.parametrize("gen", ["numpy", "torch"])
def test_long_row_recipe(gen):
    N, L = 3000, 2500
    A = synth.long_row(N, L, short_len=3, at=1000, seed=5) if gen == "numpy" else \
        synth.long_row_device(N, L, short_len=3, at=1000, seed=5, device="cpu")
    _check_csr(A)
    rl = np.diff(_np(A.rpt))
    assert rl[1000] == L and np.all(np.delete(rl, 1000) == 3)


@pytest.mark.parametrize("N,C", [(16, 4), (64, 8)])
def test_beta_worst_recipe(N, C):
    A = synth.beta_worst(N, C)
    _check_csr(A)
    rl = A.row_lengths()
    assert np.all(rl[::C] == N)
    for i in range(N):
        if i % C:
            assert rl[i] == 1 and A.col[A.rpt[i]] == i


def test_dense_device_recipe():
    D = synth.dense_device(5, 7, device="cpu")
    _check_csr(D, square=False)
    assert D.nrows == 5 and D.ncols == 7 and D.nnz == 35


def test_vectors_in_range_and_seeded():
    x = synth.vector(10_000, seed=3)
    assert x.min() >= -1 and x.max() < 1 and abs(x.mean()) < 0.03
    assert np.array_equal(x, synth.vector(10_000, seed=3))
    assert not np.array_equal(x, synth.vector(10_000, seed=4))
    X = synth.block(100, 8, seed=1)
    assert X.shape == (100, 8) and X.flags["C_CONTIGUOUS"]
