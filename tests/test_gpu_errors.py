"""Failure handling through the C ABI, made on the host: malformed CRS input,
bad options, and an allocator that fails on demand (no GPU fault involved)."""

import numpy as np
import pytest

from paper_1307_6209_gb300 import synth

pytestmark = pytest.mark.gpu


def _status(fn, *a, **k):
    from paper_1307_6209_gb300 import sell
    try:
        fn(*a, **k)
    except sell.SellError as e:
        return e.status
    return sell.SELL_OK


def test_malformed_csr_is_einval():
    import torch
    from paper_1307_6209_gb300 import sell

    A = synth.lognormal(500, seed=1, cap=50)
    bad = []
    B = synth.CSR(A.nrows, A.ncols, A.rpt.copy(), A.col.copy(), A.val)
    B.rpt[0] = 1
    bad.append(B)
    B = synth.CSR(A.nrows, A.ncols, A.rpt.copy(), A.col.copy(), A.val)
    B.rpt[10], B.rpt[11] = B.rpt[11], B.rpt[10]  # decreasing somewhere
    bad.append(B)
    B = synth.CSR(A.nrows, A.ncols, A.rpt.copy(), A.col.copy(), A.val)
    B.col[7] = A.ncols  # out of range
    bad.append(B)
    B = synth.CSR(A.nrows, A.ncols, A.rpt.copy(), A.col.copy(), A.val)
    B.col[3] = -1
    bad.append(B)
    for B in bad:
        assert _status(sell.sell_build, B, C=32, sigma=64) == sell.SELL_EINVAL
        Bd = synth.CSR(B.nrows, B.ncols, torch.from_numpy(B.rpt).cuda(), torch.from_numpy(B.col).cuda(),
                       torch.from_numpy(B.val).cuda())
        assert _status(sell.sell_build, Bd, C=32, sigma=64) == sell.SELL_EINVAL
    assert "malformed" in sell.sell_last_error() or "rpt" in sell.sell_last_error()


def test_bad_options_are_einval():
    from paper_1307_6209_gb300 import sell

    A = synth.random_csr(40, 30, density=0.2, seed=0)
    assert _status(sell.sell_build, A, C=0) == sell.SELL_EINVAL
    assert _status(sell.sell_build, A, C=32, sigma=0) == sell.SELL_EINVAL
    assert _status(sell.sell_build, A, C=32, store_type=9) == sell.SELL_EINVAL
    assert _status(sell.sell_build, A, C=32, flags=sell.SELL_BUILD_PERMUTE_COLS) == sell.SELL_EINVAL
    assert _status(sell.sell_build, A, C=32, flags=0x80) == sell.SELL_EINVAL
    h = sell.sell_build(synth.laplace2d(8), C=32)
    assert _status(sell.sell_set_launch, h, 48, 0) == sell.SELL_EINVAL
    assert _status(sell.sell_set_launch, h, 0, 3) == sell.SELL_EINVAL
    assert _status(sell.sell_set_launch, h, 0, 0, 3) == sell.SELL_EINVAL
    h1 = sell.sell_build(synth.laplace2d(8), C=16)
    assert _status(sell.sell_set_launch, h1, 0, 0, 2) == sell.SELL_EUNSUPPORTED
    sell.sell_check(h1)  # nothing pending, no bounded wait gave up
    assert _status(sell.sell_set_launch, h, 0, 0, -2) == sell.SELL_EINVAL
    lib = sell.load()
    assert lib.sell_spmmv(h.handle, None, 1, None, 1, 0, 0, None) == sell.SELL_EINVAL
    assert lib.sell_spmv(None, None, None, 0, None) == sell.SELL_EINVAL
    assert lib.sell_free(None) == sell.SELL_OK


def test_failing_allocator_reports_enomem_without_leak():
    """An allocator that fails at the n-th request: sell_build must return
    SELL_ENOMEM and give back every buffer it obtained."""
    import torch
    from paper_1307_6209_gb300 import sell

    lib = sell.load()
    A = synth.lognormal(20000, seed=2, cap=500)
    live = set()
    state = {"n": 0, "fail_at": -1}

    def _alloc(nbytes, ctx, stream):
        state["n"] += 1
        if state["n"] == state["fail_at"]:
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)
        live.add(p)
        return p

    def _free(ptr, ctx, stream):
        if ptr:
            live.discard(ptr)
            torch.cuda.caching_allocator_delete(ptr)

    a, f = sell.ALLOC_FN(_alloc), sell.FREE_FN(_free)
    assert lib.sell_set_allocator(a, f, None) == sell.SELL_OK
    try:
        # count the requests of a successful build (radix path: many buffers)
        state["fail_at"] = -1
        state["n"] = 0
        h = sell.sell_build(A, C=32, sigma=8192)
        total = state["n"]
        h.free()
        torch.cuda.synchronize()
        assert not live and total >= 8
        for k in range(1, total + 1):
            state["n"] = 0
            state["fail_at"] = k
            assert _status(sell.sell_build, A, C=32, sigma=8192) == sell.SELL_ENOMEM
            torch.cuda.synchronize()
            assert not live, f"leak after failing request {k}"
    finally:
        assert lib.sell_set_allocator(sell.ALLOC_FN(), sell.FREE_FN(), None) == sell.SELL_OK


def test_binding_refuses_mismatched_buffers():
    """The Python binding checks what the C call cannot see: element type,
    host/device placement and a unit stride along the right-hand sides."""
    import numpy as np
    import torch
    from paper_1307_6209_gb300 import sell

    A = synth.laplace2d(16)
    h = sell.sell_build(A, C=32)
    x32 = torch.zeros(A.ncols, dtype=torch.float32, device="cuda")
    y = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")
    with pytest.raises(TypeError):
        sell.sell_spmv(h, x32, y)  # binary32 x for binary64 storage
    with pytest.raises(TypeError):
        sell.sell_spmv(h, np.zeros(A.ncols), np.zeros(A.nrows))  # host arrays without HOST_IO
    with pytest.raises(TypeError):
        sell.sell_spmv(h, torch.zeros(A.ncols, dtype=torch.float64, device="cuda"), np.zeros(A.nrows),
                       flags=sell.SELL_SPMV_HOST_IO)  # device x with HOST_IO
    X = torch.zeros((A.ncols, 8), dtype=torch.float64, device="cuda")
    Y = torch.zeros((A.nrows, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        sell.sell_spmmv(h, X[:, ::2], Y)  # every other column: not contiguous along k


def test_bounded_device_wait_runs_out_and_is_reported():
    """The bulk-staged SpMV's failure route, made without a fault: one warp
    waits (1 ms limit) on a barrier that nothing completes, gives up, drains
    its own copies and ends; sell_check reports SELL_ETIMEOUT once and clears
    it, and the next product -- normal limits -- is bitwise the launch-mode-0
    product again."""
    import torch
    from paper_1307_6209_gb300 import sell

    # a banded matrix with no long rows: every warp of the bulk-staged grid
    # (about five chunks each) stages pieces, the first warp included
    A = synth.banded(400_000, seed=9)
    h = sell.sell_build(A, C=32, sigma=1)
    x = torch.from_numpy(synth.vector(A.ncols, seed=2)).cuda()
    y0 = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
    sell.sell_spmv(h, x, y0)
    assert _status(sell.sell_test_expire_wait, h, 1000) == sell.SELL_EUNSUPPORTED  # launch mode 0
    sell.sell_set_launch(h, 256, 4, 2)
    assert _status(sell.sell_test_expire_wait, h, 0) == sell.SELL_EINVAL
    assert _status(sell.sell_test_expire_wait, h, 2_000_000) == sell.SELL_EINVAL
    sell.sell_test_expire_wait(h, 1000)
    y = torch.full((A.nrows,), float("nan"), dtype=torch.float64, device="cuda")
    sell.sell_spmv(h, x, y)
    assert _status(sell.sell_check, h) == sell.SELL_ETIMEOUT
    assert "gave up" in sell.sell_last_error()
    assert torch.isnan(y).any()  # the rows of the warp that gave up were never written
    sell.sell_check(h)  # the record was cleared
    y.fill_(float("nan"))
    sell.sell_spmv(h, x, y)  # the hook applied to one launch only
    sell.sell_check(h)
    assert torch.equal(y, y0)
    h.free()
