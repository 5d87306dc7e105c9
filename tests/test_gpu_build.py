"""GPU format parity: the arrays built by sell_build (CUDA) against the CPU
oracle's step-by-step build, byte for byte (Sec. 3.3-3.4)."""
import numpy as np
import pytest

import oracle
from paper_1307_6209_gb300 import synth
from tests.gpu_util import parity_matrices

pytestmark = pytest.mark.gpu

CS = [1, 2, 3, 32, 64, 128]
SIGMAS = [1, 2, 5, 32, 256, 4096, 10 ** 9]


def _compare(A, C, sigma, store=0, flags=0, on_device=False):
    import torch
    from paper_1307_6209_gb300 import sell

    if on_device:
        Ad = synth.CSR(A.nrows, A.ncols, torch.from_numpy(A.rpt).cuda(),
                       torch.from_numpy(A.col).cuda(), torch.from_numpy(A.val).cuda())
        h = sell.sell_build(Ad, C=C, sigma=sigma, store_type=store, flags=flags)
    else:
        h = sell.sell_build(A, C=C, sigma=sigma, store_type=store, flags=flags)
    G = sell.sell_export(h)
    F = oracle.sell_build(A, C, sigma, permute_cols=bool(flags & sell.SELL_BUILD_PERMUTE_COLS))
    for k in ("cs", "cl", "srl", "perm", "col"):
        assert G[k].tobytes() == F[k].tobytes(), f"{k} differs (C={C}, sigma={sigma})"
    if store == sell.SELL_F64:
        ref = F["val"]
    else:
        ref = oracle.round_values(F["val"], store)
    assert G["val"].tobytes() == ref.tobytes(), f"val differs (C={C}, sigma={sigma}, store={store})"
    inf = h.info
    assert inf.stored == F["stored"] and inf.nchunks == F["nchunks"]
    assert inf.beta == F["beta"]
    assert inf.max_row_len == (int(A.row_lengths().max()) if A.nrows else 0)
    assert inf.zeta == pytest.approx(F["zeta"], rel=1e-9, abs=1e-12)
    h.free()


@pytest.mark.parametrize("name,A", parity_matrices(), ids=lambda v: v if isinstance(v, str) else "")
@pytest.mark.parametrize("C", CS)
def test_format_bitexact_sweep(name, A, C):
    for sigma in SIGMAS:
        _compare(A, C, sigma)


@pytest.mark.parametrize("store", [1, 2])
def test_format_reduced_precision_values(store):
    """Binary32 / bfloat16 storage: one round-to-nearest-even per value."""
    A = synth.lognormal(4000, seed=7, cap=200)
    A.val = A.val * np.exp(np.random.default_rng(0).uniform(-30, 30, A.val.shape[0]))
    for C, sigma in [(32, 1), (64, 256), (7, 100)]:
        _compare(A, C, sigma, store=store)


def test_format_float32_input():
    A = synth.lognormal(2000, seed=8, cap=100)
    A32 = synth.CSR(A.nrows, A.ncols, A.rpt, A.col, A.val.astype(np.float32))
    from paper_1307_6209_gb300 import sell
    h = sell.sell_build(A32, C=32, sigma=64, store_type=sell.SELL_F64)
    G = sell.sell_export(h)
    A64 = synth.CSR(A.nrows, A.ncols, A.rpt, A.col, A.val.astype(np.float32).astype(np.float64))
    F = oracle.sell_build(A64, 32, 64)
    assert G["val"].tobytes() == F["val"].tobytes()


def test_format_device_csr_input():
    A = synth.lognormal(3000, seed=9, cap=100)
    for C, sigma in [(32, 1), (32, 512), (128, 10 ** 9)]:
        _compare(A, C, sigma, on_device=True)


def test_format_radix_sort_path():
    """Scopes above 4096 rows go through the LSD radix sort (several windows
    and several 8-bit digit passes), which must give the same stable order."""
    A = synth.lognormal(70001, seed=10, cap=2000)
    for sigma in [4097, 8192, 30000, 10 ** 9]:
        _compare(A, 32, sigma)
    # key wider than 16 bits: many windows plus long rows
    B = synth.long_row(200000, 70000, short_len=5, at=150000, seed=11)
    _compare(B, 64, 5000)


def test_format_permuted_columns():
    from paper_1307_6209_gb300 import sell
    A = synth.lognormal(3001, seed=12, cap=100)
    for C, sigma in [(32, 128), (64, 10 ** 9), (32, 1)]:
        _compare(A, C, sigma, flags=sell.SELL_BUILD_PERMUTE_COLS)


def test_format_laplace_beta_and_special_cases():
    """SELL-1-1 == CRS and the 64x64 Laplacian's beta through the GPU path."""
    from paper_1307_6209_gb300 import sell
    A = synth.laplace2d(64)
    h = sell.sell_build(A, C=1, sigma=1)
    G = sell.sell_export(h)
    assert G["val"].tobytes() == A.val.tobytes() and np.array_equal(G["cs"], A.rpt)
    h = sell.sell_build(A, C=32, sigma=1)
    assert h.info.beta == 20224 / 20352
    # sigma = 4096 sorts the whole grid: 3844 rows of length 5, 248 of 4, 4 of
    # 3 -> 120 full chunks of width 5, one mixed chunk of width 5, then 7
    # chunks of width 4: 32 * (121 * 5 + 7 * 4) = 20256 stored elements
    h = sell.sell_build(A, C=32, sigma=4096)
    assert h.info.beta == 20224 / 20256
