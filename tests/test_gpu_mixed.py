"""Reduced-precision storage (binary32 / bfloat16 values, binary32 x and
accumulation) against the binary64 oracle evaluated on the same rounded
values and the same binary32 x.  Bounds: tests/gpu_util.tol_f32 (plain FMA
chain) and tol_dot2 (compensated).  The error against the unrounded binary64
product is reported as well (it is dominated by the value rounding)."""
import numpy as np
import pytest

import oracle
from paper_1307_6209_gb300 import synth
from tests.gpu_util import tol_dot2, tol_f32

pytestmark = pytest.mark.gpu


def _rounded(A, store):
    r = oracle.round_values(A.val, store)
    v = r.astype(np.float64) if store == 1 else oracle.bf16_to_f64(r)
    return synth.CSR(A.nrows, A.ncols, A.rpt, A.col, v)


@pytest.mark.parametrize("store", [1, 2])
@pytest.mark.parametrize("comp", [False, True, "long"])
@pytest.mark.parametrize("k", [1, 4, 8])
def test_mixed_precision_within_bound(store, comp, k):
    import torch
    from paper_1307_6209_gb300 import sell

    A = synth.lognormal(6000, seed=store * 10 + k, cap=1500)
    Ar = _rounded(A, store)
    X = synth.block(A.ncols, k, seed=k).astype(np.float32)
    h = sell.sell_build(A, C=32, sigma=512, store_type=store)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.empty((A.nrows, k), dtype=torch.float32, device="cuda")
    flags = {False: 0, True: sell.SELL_SPMV_COMPENSATED, "long": sell.SELL_SPMV_COMPENSATED_LONG}[comp]
    sell.sell_spmmv(h, Xd, Yd, flags=flags)
    torch.cuda.synchronize()
    Y = Yd.cpu().numpy().astype(np.float64)
    rl = A.row_lengths()
    for c in range(k):
        x64 = X[:, c].astype(np.float64)
        ref = oracle.csr_spmv(Ar, x64)
        scale = oracle.csr_absdot(Ar, x64)
        if comp == "long":  # Dot2 on rows of more than 64 entries, binary32 chains on the others
            tol = np.where(rl > 64, tol_dot2(rl, scale, ref), tol_f32(rl, scale))
        else:
            tol = tol_dot2(rl, scale, ref) if comp else tol_f32(rl, scale)
        assert np.all(np.abs(Y[:, c] - ref) <= tol), f"column {c}"
    if comp is True:
        # compensated results are the rounded exact sums up to ~gamma_n^2
        rel = np.abs(Y[:, 0] - oracle.csr_spmv(Ar, X[:, 0].astype(np.float64)))
        assert np.median(rel / np.maximum(oracle.csr_absdot(Ar, X[:, 0].astype(np.float64)), 1e-300)) < 2 ** -24


def test_compensated_on_f64_is_unsupported():
    import torch
    from paper_1307_6209_gb300 import sell

    A = synth.laplace2d(16)
    h = sell.sell_build(A, C=32, sigma=1)
    x = torch.ones(A.ncols, dtype=torch.float64, device="cuda")
    y = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
    with pytest.raises(sell.SellError) as e:
        sell.sell_spmv(h, x, y, flags=sell.SELL_SPMV_COMPENSATED)
    assert e.value.status == sell.SELL_EUNSUPPORTED


def test_mixed_invariant_across_formats():
    """The binary32 chain is also bitwise independent of (C, sigma) and of the
    launch shape (block, unroll, software pipelining)."""
    import torch
    from paper_1307_6209_gb300 import sell

    A = synth.lognormal(5000, seed=3, cap=400)
    x = torch.from_numpy(synth.vector(A.ncols, seed=1).astype(np.float32)).cuda()
    outs = []
    for C, sigma in [(32, 1), (64, 4096), (128, 10 ** 9)]:
        for store in (1, 2):
            h = sell.sell_build(A, C=C, sigma=sigma, store_type=store)
            y = torch.empty(A.nrows, dtype=torch.float32, device="cuda")
            for fl in (0, sell.SELL_SPMV_COMPENSATED, sell.SELL_SPMV_COMPENSATED_LONG):
                for block, unroll, pipe in ((256, 4, 0), (128, 8, 1), (512, 1, 1), (256, 2, 2), (128, 8, 2)):
                    sell.sell_set_launch(h, block, unroll, pipe)
                    sell.sell_spmv(h, x, y, flags=fl)
                    torch.cuda.synchronize()
                    outs.append(((store, fl), y.cpu().numpy().tobytes()))
    by = {}
    for key, b in outs:
        by.setdefault(key, set()).add(b)
    assert all(len(v) == 1 for v in by.values())
