"""sell_spmmv_noalloc: the product for callers that cannot allocate device
memory while they multiply (a serving loop held to a fixed memory budget,
code inside another framework's memory pool, a latency-critical path).  It
must give the same results as sell_spmmv, call after call, while keeping the
long-row scratch in the library's fixed 4 MiB device array.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  It also passes when run
alone in a fresh process."""
import ctypes

import numpy as np
import pytest

from paper_1307_6209_gb300 import synth
from tests.gpu_util import assert_oracle_parity

pytestmark = pytest.mark.gpu


def _noalloc(h, X, Y, flags=0):
    """Call the C entry point directly through the ABI."""
    from paper_1307_6209_gb300 import sell
    import torch
    lib = sell.load()
    if X.dim() == 1:
        k, ldx, ldy = 1, 1, 1
    else:
        k, ldx, ldy = X.shape[1], X.stride(0), Y.stride(0)
    return lib.sell_spmmv_noalloc(h.handle, ctypes.c_void_p(X.data_ptr()), ldx, ctypes.c_void_p(Y.data_ptr()),
                                  ldy, k, flags, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _rows_of_65(N, seed=0):
    """N rows of 65 entries each (two segments per row), cheap to generate."""
    i = np.arange(N, dtype=np.int64)[:, None]
    col = np.sort((i + np.arange(65, dtype=np.int64)[None, :] * 37) % N, axis=1).astype(np.int32).ravel()
    rpt = np.arange(N + 1, dtype=np.int64) * 65
    val = np.random.default_rng(seed).standard_normal(col.shape[0])
    return synth.CSR(N, N, rpt, col, val)


@pytest.mark.parametrize("k,pad", [(1, 0), (5, 3), (8, 0)])
def test_noalloc_matches_spmmv_twice(k, pad):
    import torch
    from paper_1307_6209_gb300 import sell

    A = synth.lognormal(20000, seed=21, cap=2000)  # many rows longer than 64 entries
    h = sell.sell_build(A, C=32, sigma=A.nrows)
    assert h.info.nrows == A.nrows
    for call in range(2):  # two calls in a row: the shared array keeps old contents
        X = synth.block(A.ncols, k, seed=100 + call)
        Xd = torch.zeros((A.ncols, k + pad), dtype=torch.float64, device="cuda")
        Xd[:, :k] = torch.from_numpy(X).cuda()
        Yref = torch.full((A.nrows, k + pad), float("nan"), dtype=torch.float64, device="cuda")
        Ynew = torch.full((A.nrows, k + pad), float("nan"), dtype=torch.float64, device="cuda")
        if k == 1 and pad == 0:
            xs, yr, yn = Xd[:, 0].contiguous(), Yref[:, 0].contiguous(), Ynew[:, 0].contiguous()
            sell.sell_spmmv(h, xs, yr, ldx=1, ldy=1, k=1)
            assert _noalloc(h, xs, yn) == sell.SELL_OK, sell.sell_last_error()
            torch.cuda.synchronize()
            ref, new = yr.cpu().numpy()[:, None], yn.cpu().numpy()[:, None]
        else:
            sell.sell_spmmv(h, Xd[:, :k], Yref[:, :k])
            assert _noalloc(h, Xd[:, :k], Ynew[:, :k]) == sell.SELL_OK, sell.sell_last_error()
            torch.cuda.synchronize()
            ref, new = Yref[:, :k].cpu().numpy(), Ynew[:, :k].cpu().numpy()
            if pad:
                assert torch.isnan(Ynew[:, k:]).all()
        # against the oracle's binary64 CRS product, within the binary64 bound
        assert_oracle_parity(A, sell.SELL_F64, X, new, what=f"call {call}")
        # the same per-row arithmetic runs in both entry points
        assert new.tobytes() == ref.tobytes()


def test_noalloc_compensated_f32_twice():
    import torch
    from paper_1307_6209_gb300 import sell

    A = synth.lognormal(15000, seed=22, cap=1500)
    h = sell.sell_build(A, C=64, sigma=4096, store_type=sell.SELL_F32)
    for call in range(2):
        x = torch.from_numpy(synth.vector(A.ncols, seed=call).astype(np.float32)).cuda()
        y0 = torch.from_numpy(synth.vector(A.nrows, seed=50 + call).astype(np.float32)).cuda()
        yr, yn = y0.clone(), y0.clone()
        fl = sell.SELL_SPMV_COMPENSATED | sell.SELL_SPMV_ACCUMULATE
        sell.sell_spmv(h, x, yr, flags=fl)
        assert _noalloc(h, x, yn, flags=fl) == sell.SELL_OK, sell.sell_last_error()
        torch.cuda.synchronize()
        ref, new = yr.cpu().numpy(), yn.cpu().numpy()
        # against the oracle on the binary32-rounded values, within the Dot2 bound
        assert_oracle_parity(A, sell.SELL_F32, x.cpu().numpy(), new, flags=fl, Y0=y0.cpu().numpy(),
                             what=f"call {call}")
        assert new.tobytes() == ref.tobytes()


def test_noalloc_rejects_what_it_cannot_do():
    import torch
    from paper_1307_6209_gb300 import sell

    # 300,000 rows of 65 entries: one column of long-row scratch needs
    # 18,750 units x 32 lanes x 8 bytes = 4.8 MB, more than the 4 MiB array
    A = _rows_of_65(300000)
    h = sell.sell_build(A, C=32, sigma=1)
    x = torch.ones(A.ncols, dtype=torch.float64, device="cuda")
    y = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
    assert _noalloc(h, x, y) == sell.SELL_EINVAL
    assert "scratch" in sell.sell_last_error()
    # host buffers would need staging memory
    B = synth.laplace2d(32)
    hb = sell.sell_build(B, C=32, sigma=1)
    xh = np.ones(B.ncols)
    yh = np.zeros(B.nrows)
    lib = sell.load()
    st = lib.sell_spmmv_noalloc(hb.handle, ctypes.c_void_p(xh.ctypes.data), 1, ctypes.c_void_p(yh.ctypes.data),
                                1, 1, sell.SELL_SPMV_HOST_IO, None)
    assert st == sell.SELL_EINVAL
    # a smaller matrix of the same kind fits and matches sell_spmv
    S = _rows_of_65(40000, seed=1)
    hs = sell.sell_build(S, C=32, sigma=1)
    xs = torch.from_numpy(synth.vector(S.ncols, seed=3)).cuda()
    ya = torch.empty(S.nrows, dtype=torch.float64, device="cuda")
    yb = torch.empty(S.nrows, dtype=torch.float64, device="cuda")
    sell.sell_spmv(hs, xs, ya)
    assert _noalloc(hs, xs, yb) == sell.SELL_OK, sell.sell_last_error()
    torch.cuda.synchronize()
    assert torch.equal(ya, yb)
    assert_oracle_parity(S, sell.SELL_F64, xs.cpu().numpy(), yb.cpu().numpy(), what="40000 rows of 65")
    # eight columns do not fit there (the array holds four): the columns run
    # in narrower blocks, and k = 5 with padded rows leaves the padding alone
    for k, pad in ((8, 0), (5, 3)):
        X = synth.block(S.ncols, k, seed=40 + k)
        Xd = torch.full((S.ncols, k + pad), 9.0, dtype=torch.float64, device="cuda")
        Xd[:, :k] = torch.from_numpy(X).cuda()
        Yr = torch.full((S.nrows, k + pad), -1.5, dtype=torch.float64, device="cuda")
        Yn = Yr.clone()
        sell.sell_spmmv(hs, Xd[:, :k], Yr[:, :k])
        assert _noalloc(hs, Xd[:, :k], Yn[:, :k]) == sell.SELL_OK, sell.sell_last_error()
        torch.cuda.synchronize()
        assert Yn.cpu().numpy().tobytes() == Yr.cpu().numpy().tobytes()
        assert torch.all(Yn[:, k:] == -1.5)
        assert_oracle_parity(S, sell.SELL_F64, X, Yn[:, :k].cpu().numpy(), what=f"k={k}")
