"""Parity at the full sizes of the benchmark configurations, in the launch
configuration bench.py times (tuned C, sigma, block, unroll):

* lognormal random N = 2,000,000 (~32 M nnz): every format array byte for
  byte against the oracle's build, y for every row against the oracle's CRS
  product within the binary64 row-wise bound;
* 27-point stencil on 200^3 (213,847,192 nnz = 598^3): chunk structure and
  row lengths byte for byte, the stored size against its closed form, every
  y against the oracle; binary32 and bfloat16 storage within the binary32
  bound against the oracle on the rounded values.
"""
import numpy as np
import pytest

import oracle
from paper_1307_6209_gb300 import synth
from tests.gpu_util import tol_f32, tol_f64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lognormal2m():
    return synth.lognormal(2_000_000, mean=16.0, sigma_ln=1.2, cap=2000, seed=0)


@pytest.mark.parametrize("C,sigma,block,unroll,pipe", [(64, 2_000_000, 128, 4, 1), (32, 2_000_000, 128, 8, 0),
                                                       (32, 1, 256, 4, 1), (128, 4096, 128, 2, 0),
                                                       (32, 2_000_000, 256, 2, 2), (128, 2_000_000, 512, 4, 2),
                                                       (128, 2_000_000, 512, 1, 2)])
def test_lognormal_2m_full(lognormal2m, C, sigma, block, unroll, pipe):
    import torch
    from paper_1307_6209_gb300 import sell

    A = lognormal2m
    h = sell.sell_build(A, C=C, sigma=sigma)
    G = sell.sell_export(h)
    F = oracle.sell_build(A, C, sigma)
    for k in ("cs", "cl", "srl", "perm", "col", "val"):
        assert G[k].tobytes() == F[k].tobytes(), k
    sell.sell_set_launch(h, block, unroll, pipe)
    x = synth.vector(A.ncols, seed=0)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
    sell.sell_spmv(h, xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    ref = oracle.csr_spmv(A, x, nthreads=0, guided=True)
    scale = oracle.csr_absdot(A, x)
    assert np.all(np.abs(y - ref) <= tol_f64(A.row_lengths(), scale))
    h.free()


def test_stencil27_200_full():
    import torch
    from paper_1307_6209_gb300 import sell

    n = 200
    Ad = synth.stencil27_device(n, perturb=0.1, seed=0)
    A = synth.CSR(Ad.nrows, Ad.ncols, Ad.rpt.cpu().numpy(), Ad.col.cpu().numpy(), Ad.val.cpu().numpy())
    assert A.nnz == (3 * n - 2) ** 3 == 213_847_192
    h = sell.sell_build(Ad, C=32, sigma=1)
    sell.sell_set_launch(h, 128, 4, 1)
    x = synth.vector(A.ncols, seed=0)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
    sell.sell_spmv(h, xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    ref = oracle.csr_spmv(A, x, nthreads=0)
    scale = oracle.csr_absdot(A, x)
    assert np.all(np.abs(y - ref) <= tol_f64(A.row_lengths(), scale))
    # the bulk-staged launch mode gives the same bits at full size
    sell.sell_set_launch(h, 256, 4, 2)
    yb = torch.full((A.nrows,), float("nan"), dtype=torch.float64, device="cuda")
    sell.sell_spmv(h, xd, yb)
    sell.sell_check(h)
    assert yb.cpu().numpy().tobytes() == y.tobytes()
    del yb

    # structure: SELL-32-1 keeps the original order; the chunk widths are the
    # longest row of every 32 consecutive rows (Eq. "max")
    G = sell.sell_export(h)
    rl = A.row_lengths()
    npad = (-A.nrows) % 32
    cl = np.concatenate([rl, np.zeros(npad, rl.dtype)]).reshape(-1, 32).max(1)
    assert np.array_equal(G["cl"], cl)
    assert np.array_equal(G["srl"][:A.nrows], rl) and np.array_equal(G["perm"], np.arange(A.nrows))
    assert G["cs"][-1] == 32 * int(cl.sum()) == h.info.stored
    # spot-check stored entries of a few chunks against the CRS arrays
    rng = np.random.default_rng(0)
    for c in rng.integers(0, cl.shape[0], 200):
        for l in (0, 13, 31):
            r = int(c) * 32 + l
            if r >= A.nrows:
                continue
            j = np.arange(rl[r])
            pos = G["cs"][c] + j * 32 + l
            assert np.array_equal(G["col"][pos], A.col[A.rpt[r]:A.rpt[r + 1]])
            assert np.array_equal(G["val"][pos], A.val[A.rpt[r]:A.rpt[r + 1]])
    del G
    h.free()

    # binary32 storage at full size: within the binary32 FMA-chain bound
    h32 = sell.sell_build(Ad, C=32, sigma=1, store_type=sell.SELL_F32)
    sell.sell_set_launch(h32, 128, 8, 1)
    x32 = x.astype(np.float32)
    y32 = torch.empty(A.nrows, dtype=torch.float32, device="cuda")
    sell.sell_spmv(h32, torch.from_numpy(x32).cuda(), y32)
    torch.cuda.synchronize()
    Ar = synth.CSR(A.nrows, A.ncols, A.rpt, A.col, oracle.round_values(A.val, oracle.F32).astype(np.float64))
    x64 = x32.astype(np.float64)
    ref32 = oracle.csr_spmv(Ar, x64, nthreads=0)
    scale32 = oracle.csr_absdot(Ar, x64)
    assert np.all(np.abs(y32.cpu().numpy().astype(np.float64) - ref32) <= tol_f32(rl, scale32))
    h32.free()
    del Ar, ref32, scale32

    # bfloat16 storage at full size (the benchmark's bf16 stencil), same x
    hb = sell.sell_build(Ad, C=32, sigma=1, store_type=sell.SELL_BF16)
    sell.sell_set_launch(hb, 256, 4, 1)
    sell.sell_spmv(hb, torch.from_numpy(x32).cuda(), y32)
    torch.cuda.synchronize()
    Ab = synth.CSR(A.nrows, A.ncols, A.rpt, A.col, oracle.bf16_to_f64(oracle.round_values(A.val, oracle.BF16)))
    refb = oracle.csr_spmv(Ab, x64, nthreads=0)
    scaleb = oracle.csr_absdot(Ab, x64)
    assert np.all(np.abs(y32.cpu().numpy().astype(np.float64) - refb) <= tol_f32(rl, scaleb))
    hb.free()
