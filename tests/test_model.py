"""Pins of the performance model (Sec. 4) against the values the paper prints."""
import os

import pytest

from paper_1307_6209_gb300 import model

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_best_bound.txt")


def _rows():
    for ln in open(GOLDEN):
        if ln.strip() and not ln.startswith("#"):
            name, copy_bw, read_bw, bound = ln.split()
            yield name, float(copy_bw), float(read_bw), float(bound)


@pytest.mark.parametrize("name,copy_bw,read_bw,bound", list(_rows()))
def test_best_bound_matches_printed_values(name, copy_bw, read_bw, bound):
    """Sec. 5.2: P = b beta / 6 with the best of the two bandwidths of Table
    "tab:architectures" gives 7.2 / 27.5 / 25.2 GF/s."""
    b = max(copy_bw, read_bw)
    assert round(model.best_bound(b, 1.0), 1) == bound
    # Eq. "roof_general" with alpha = 1/Nnzc and Nnzr -> infinity is the same bound
    assert model.roofline(b, model.balance_sell(0.0, 1.0, 1e300)) == pytest.approx(b / 6)


def test_crs_is_sell_with_beta_one():
    """Sec. 4: the CRS values follow from the SELL model with beta = 1."""
    for a in (0.0, 0.14, 1.0, 8.0):
        for nnzr in (3.11, 16.0, 98.16):
            assert model.balance_crs(a, nnzr) == model.balance_sell(a, 1.0, nnzr)


def test_alpha_inversion_round_trip():
    """Eq. "eq:sellalpha" inverts Eq. "sellbalance" for a volume V = B * 2 Nnz."""
    nnz, nnzr = 10 ** 7, 16.0
    for alpha in (0.0, 1 / 16, 0.5, 2.0):
        for beta in (0.14, 0.8, 1.0):
            v = model.balance_sell(alpha, beta, nnzr) * 2 * nnz
            assert model.alpha_from_volume(v, nnz, beta, nnzr) == pytest.approx(alpha, abs=1e-12)


def test_algorithmic_bytes_counts():
    b = model.algorithmic_bytes(nrows=100, ncols=100, nnz=1000, nchunks=4, C=32, value_bytes=8,
                                x_bytes=8, has_perm=True)
    assert b == 12 * 1000 + 800 + 800 + 4 * 128 + 400 + 8 * 5
