"""sell_spmv_dot: y = A x followed by x . y in binary64 in a fixed order.

The dot is checked against the correctly rounded sum of the products
(math.fsum) of x and the GPU's own y: a chain of n fused multiply-adds and
pairwise tree additions is within gamma_n * sum |x_i y_i| of it.  Its bits
must not depend on (C, sigma), the launch shape or the run."""
import math

import numpy as np
import pytest

import oracle
from paper_1307_6209_gb300 import synth
from tests.gpu_util import U32, U64, gamma, tol_f64

pytestmark = pytest.mark.gpu


def _run(h, x, dtype, y0=None, flags=0):
    import torch
    from paper_1307_6209_gb300 import sell
    xd = torch.from_numpy(x.astype(dtype)).cuda()
    yd = torch.from_numpy(y0.astype(dtype)).cuda() if y0 is not None else \
        torch.empty(h.info.nrows, dtype=xd.dtype, device="cuda")
    dot = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    sell.sell_spmv_dot(h, xd, yd, dot, flags=flags)
    torch.cuda.synchronize()
    return yd.cpu().numpy(), float(dot.item())


@pytest.mark.parametrize("name,A", [("laplace64", synth.laplace2d(64)),
                                    ("lognormal", synth.lognormal(20000, seed=3, cap=500)),
                                    ("long_row", synth.long_row(9000, 9000, short_len=4, at=10, seed=2))],
                         ids=lambda v: v if isinstance(v, str) else "")
def test_dot_bound_and_invariance(name, A):
    from paper_1307_6209_gb300 import sell
    x = synth.vector(A.ncols, seed=1)
    bits = set()
    for C, sigma, block, unroll, mode in [(32, 1, 256, 4, 0), (64, 10 ** 9, 128, 8, 1), (128, 256, 512, 2, 2),
                                          (1, 1, 64, 1, 0)]:
        h = sell.sell_build(A, C=C, sigma=sigma)
        try:
            sell.sell_set_launch(h, block, unroll, mode)
        except sell.SellError:
            sell.sell_set_launch(h, block, unroll, 0)
        y, d = _run(h, x, np.float64)
        n = A.nrows
        exact = math.fsum((x * y).tolist())
        assert abs(d - exact) <= gamma(n + 1, U64) * float(np.sum(np.abs(x * y))) + 1e-300
        ref = oracle.csr_spmv(A, x)
        scale = oracle.csr_absdot(A, x)
        assert np.all(np.abs(y - ref) <= tol_f64(A.row_lengths(), scale))
        bits.add(np.float64(d).tobytes())
        h.free()
    assert len(bits) == 1, "the dot depends on the format or the launch"


def test_dot_f32_accumulate_and_errors():
    import torch
    from paper_1307_6209_gb300 import sell
    A = synth.lognormal(7001, seed=4, cap=300)
    x = synth.vector(A.ncols, seed=5)
    y0 = synth.vector(A.nrows, seed=6)
    h = sell.sell_build(A, C=32, sigma=512, store_type=sell.SELL_F32)
    y, d = _run(h, x, np.float32, y0=y0, flags=sell.SELL_SPMV_ACCUMULATE)
    x32 = x.astype(np.float32).astype(np.float64)
    exact = math.fsum((x32 * y.astype(np.float64)).tolist())
    assert abs(d - exact) <= gamma(A.nrows + 1, U64) * float(np.sum(np.abs(x32 * y))) + 1e-300
    # y itself: y0 + A x in binary32 (bound of the binary32 chain with one more term)
    Ar = synth.CSR(A.nrows, A.ncols, A.rpt, A.col, oracle.round_values(A.val, oracle.F32).astype(np.float64))
    ref = oracle.csr_spmv(Ar, x32, y0=y0.astype(np.float32).astype(np.float64), accumulate=True)
    scale = oracle.csr_absdot(Ar, x32) + np.abs(y0)
    assert np.all(np.abs(y - ref) <= 1.01 * gamma(A.row_lengths() + 2, U32) * scale + 2.0 ** -140)
    dot = torch.zeros(1, dtype=torch.float64, device="cuda")
    rect = sell.sell_build(synth.random_csr(50, 40, density=0.2, seed=1), C=32)
    xd = torch.zeros(40, dtype=torch.float64, device="cuda")
    yd = torch.zeros(50, dtype=torch.float64, device="cuda")
    with pytest.raises(sell.SellError) as e:
        sell.sell_spmv_dot(rect, xd, yd, dot)
    assert e.value.status == sell.SELL_EINVAL
