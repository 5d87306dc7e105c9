"""GPU SpMV / SpMMV parity against the CPU oracle (binary64 storage).

y must agree with Listing "crs" (binary64, CRS order, no FMA) within the
row-wise bound of tests/gpu_util.tol_f64; results of the CUDA path must be
bitwise identical across (C, sigma), launch shapes and right-hand-side
blocking, because every row is one FMA chain in CRS order.
"""
import numpy as np
import pytest

import oracle
from paper_1307_6209_gb300 import synth
from tests.gpu_util import oracle_reference, parity_matrices, tol_f64

pytestmark = pytest.mark.gpu


def _spmv(h, x, y0=None, flags=0):
    import torch
    from paper_1307_6209_gb300 import sell

    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    if y0 is None:
        yd = torch.full((h.info.nrows,), float("nan"), dtype=torch.float64, device="cuda")
    else:
        yd = torch.from_numpy(np.ascontiguousarray(y0)).cuda()
    sell.sell_spmv(h, xd, yd, flags=flags)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


@pytest.mark.parametrize("name,A", parity_matrices(), ids=lambda v: v if isinstance(v, str) else "")
def test_spmv_matches_oracle_and_is_invariant(name, A):
    from paper_1307_6209_gb300 import sell

    x = synth.vector(A.ncols, seed=0)
    ref, scale, rl = oracle_reference(A, x)
    first = None
    for C, sigma in [(32, 1), (1, 1), (2, 7), (32, 256), (64, 4096), (128, 10 ** 9), (3, 5000)]:
        h = sell.sell_build(A, C=C, sigma=sigma)
        for block, unroll, pipe in [(256, 4, 0), (128, 1, 1), (512, 8, 0), (64, 2, 1), (256, 8, 1),
                                    (256, 2, 2), (128, 8, 2), (512, 4, 2), (32, 1, 2)]:
            if pipe == 2 and C not in (32, 64, 128):
                with pytest.raises(sell.SellError) as e:
                    sell.sell_set_launch(h, block, unroll, pipe)
                assert e.value.status == sell.SELL_EUNSUPPORTED
                continue
            sell.sell_set_launch(h, block, unroll, pipe)
            y = _spmv(h, x)
            sell.sell_check(h)
            assert np.all(np.abs(y - ref) <= tol_f64(rl, scale)), (C, sigma, block, unroll, pipe)
            if first is None:
                first = y
            assert y.tobytes() == first.tobytes(), "result depends on (C, sigma) or launch shape"
        h.free()


def test_spmv_accumulate():
    from paper_1307_6209_gb300 import sell

    A = synth.lognormal(3000, seed=3, cap=200)
    x = synth.vector(A.ncols, seed=1)
    y0 = synth.vector(A.nrows, seed=2)
    ref = oracle.csr_spmv(A, x, y0=y0, accumulate=True)
    scale = oracle.csr_absdot(A, x) + np.abs(y0)
    for sigma in (1, 512):
        h = sell.sell_build(A, C=32, sigma=sigma)
        y = _spmv(h, x, y0=y0, flags=sell.SELL_SPMV_ACCUMULATE)
        assert np.all(np.abs(y - ref) <= tol_f64(A.row_lengths() + 1, scale))


def test_spmv_permuted_space():
    """With the symmetric permutation the handle maps x' = Px to y' = Py."""
    from paper_1307_6209_gb300 import sell

    A = synth.lognormal(4001, seed=4, cap=150)
    x = synth.vector(A.ncols, seed=3)
    ref, scale, rl = oracle_reference(A, x)
    h = sell.sell_build(A, C=32, sigma=1024, flags=sell.SELL_BUILD_PERMUTE_COLS)
    perm = sell.sell_export(h)["perm"]
    yp = _spmv(h, x[perm])
    assert np.all(np.abs(yp - ref[perm]) <= tol_f64(rl[perm], scale[perm]))


def test_spmv_host_io():
    """HOST_IO: numpy in, numpy out; the library stages the copies."""
    from paper_1307_6209_gb300 import sell
    import torch

    A = synth.lognormal(5000, seed=5, cap=100)
    x = synth.vector(A.ncols, seed=4)
    ref, scale, rl = oracle_reference(A, x)
    h = sell.sell_build(A, C=32, sigma=256)
    y = np.full(A.nrows, np.nan)
    for _ in range(2):
        sell.sell_spmv(h, x, y, flags=sell.SELL_SPMV_HOST_IO)
        torch.cuda.synchronize()
        assert np.all(np.abs(y - ref) <= tol_f64(rl, scale))
    assert y.tobytes() == _spmv(h, x).tobytes()


@pytest.mark.parametrize("k", [1, 4, 8])
@pytest.mark.parametrize("accumulate", [False, True])
def test_spmmv_host_io_leading_dimensions(k, accumulate):
    """HOST_IO SpMMV with padded rows (ldx = ldy = k + 3) in pinned host
    memory: only the k used columns of X are read and of Y written -- the
    padding columns keep the caller's values -- every column matches the
    oracle within the binary64 bound, and the result equals the same product
    on device buffers bit for bit."""
    import torch
    from paper_1307_6209_gb300 import sell

    A = synth.lognormal(7001, seed=30 + k, cap=700)  # long rows use the segment scratch too
    h = sell.sell_build(A, C=32, sigma=4096)
    ld = k + 3
    X = synth.block(A.ncols, k, seed=7)
    Y0 = synth.block(A.nrows, k, seed=8)
    Xh = torch.full((A.ncols, ld), 7.0, dtype=torch.float64).pin_memory()
    Xh[:, :k] = torch.from_numpy(X)
    Yh = torch.full((A.nrows, ld), -3.25, dtype=torch.float64).pin_memory()
    if accumulate:
        Yh[:, :k] = torch.from_numpy(Y0)
    fl = sell.SELL_SPMV_HOST_IO | (sell.SELL_SPMV_ACCUMULATE if accumulate else 0)
    sell.sell_spmmv(h, Xh[:, :k], Yh[:, :k], flags=fl)
    torch.cuda.synchronize()
    got = Yh.numpy()
    assert np.all(got[:, k:] == -3.25), "padding columns of Y were written"
    ref = oracle.csr_spmmv(A, X, Y0=Y0 if accumulate else None, accumulate=accumulate)
    rl = A.row_lengths()
    for c in range(k):
        scale = oracle.csr_absdot(A, X[:, c]) + (np.abs(Y0[:, c]) if accumulate else 0.0)
        assert np.all(np.abs(got[:, c] - ref[:, c]) <= tol_f64(rl + (1 if accumulate else 0), scale)), f"col {c}"
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y0).cuda() if accumulate else torch.empty((A.nrows, k), dtype=torch.float64,
                                                                     device="cuda")
    sell.sell_spmmv(h, Xd, Yd, flags=fl & ~sell.SELL_SPMV_HOST_IO)
    torch.cuda.synchronize()
    assert np.ascontiguousarray(got[:, :k]).tobytes() == Yd.cpu().numpy().tobytes()


@pytest.mark.parametrize("k", [1, 4])
@pytest.mark.parametrize("accumulate", [False, True])
def test_spmmv_host_direct(k, accumulate):
    """HOST_DIRECT: the kernels read X from and write Y to page-locked host
    memory in place (padded rows, ld = k + 3): the padding keeps the caller's
    values, every column matches the oracle, and the result is the device
    product bit for bit.  Pageable host memory is refused."""
    import torch
    from paper_1307_6209_gb300 import sell

    A = synth.lognormal(6007, seed=50 + k, cap=900)
    h = sell.sell_build(A, C=64, sigma=1024)
    ld = k + 3
    X = synth.block(A.ncols, k, seed=17)
    Y0 = synth.block(A.nrows, k, seed=18)
    Xh = torch.full((A.ncols, ld), 5.0, dtype=torch.float64).pin_memory()
    Xh[:, :k] = torch.from_numpy(X)
    Yh = torch.full((A.nrows, ld), -2.5, dtype=torch.float64).pin_memory()
    if accumulate:
        Yh[:, :k] = torch.from_numpy(Y0)
    fl = sell.SELL_SPMV_HOST_DIRECT | (sell.SELL_SPMV_ACCUMULATE if accumulate else 0)
    sell.sell_spmmv(h, Xh[:, :k], Yh[:, :k], flags=fl)
    torch.cuda.synchronize()
    got = Yh.numpy()
    assert np.all(got[:, k:] == -2.5), "padding columns of Y were written"
    ref = oracle.csr_spmmv(A, X, Y0=Y0 if accumulate else None, accumulate=accumulate)
    rl = A.row_lengths()
    for c in range(k):
        scale = oracle.csr_absdot(A, X[:, c]) + (np.abs(Y0[:, c]) if accumulate else 0.0)
        assert np.all(np.abs(got[:, c] - ref[:, c]) <= tol_f64(rl + (1 if accumulate else 0), scale)), f"col {c}"
    Yd = torch.from_numpy(Y0).cuda() if accumulate else torch.empty((A.nrows, k), dtype=torch.float64,
                                                                     device="cuda")
    sell.sell_spmmv(h, torch.from_numpy(X).cuda(), Yd, flags=fl & ~sell.SELL_SPMV_HOST_DIRECT)
    torch.cuda.synchronize()
    assert np.ascontiguousarray(got[:, :k]).tobytes() == Yd.cpu().numpy().tobytes()
    lib = sell.load()
    xp, yp = np.ones(A.ncols), np.zeros(A.nrows)  # pageable
    assert lib.sell_spmmv(h.handle, xp.ctypes.data, 1, yp.ctypes.data, 1, 1, sell.SELL_SPMV_HOST_DIRECT,
                          None) == sell.SELL_EINVAL
    assert lib.sell_spmmv(h.handle, xp.ctypes.data, 1, yp.ctypes.data, 1, 1,
                          sell.SELL_SPMV_HOST_DIRECT | sell.SELL_SPMV_HOST_IO, None) == sell.SELL_EINVAL


def test_spmv_host_io_alternating_streams():
    """HOST_IO calls that alternate two streams (the overlapped end-to-end
    pattern): every call's y is bitwise the device-buffer product of its own
    x, including rows long enough to use the shared long-row scratch and the
    accumulate flag."""
    import torch
    from paper_1307_6209_gb300 import sell

    A = synth.lognormal(20000, seed=21, cap=3000)
    h = sell.sell_build(A, C=32, sigma=10 ** 9)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    n = 12
    xs = [torch.from_numpy(synth.vector(A.ncols, seed=100 + i)).pin_memory() for i in range(n)]
    y0 = [torch.from_numpy(synth.vector(A.nrows, seed=200 + i)).pin_memory() for i in range(n)]
    ys = [torch.full((A.nrows,), float("nan"), dtype=torch.float64).pin_memory() for _ in range(n)]
    for i in range(n):
        fl = sell.SELL_SPMV_HOST_IO | (sell.SELL_SPMV_ACCUMULATE if i % 3 == 2 else 0)
        if i % 3 == 2:
            ys[i].copy_(y0[i])
        sell.sell_spmv(h, xs[i], ys[i], flags=fl, stream=streams[i % 2])
    torch.cuda.synchronize()
    for i in range(n):
        acc = i % 3 == 2
        want = _spmv(h, xs[i].numpy(), y0=y0[i].numpy() if acc else None,
                     flags=sell.SELL_SPMV_ACCUMULATE if acc else 0)
        assert ys[i].numpy().tobytes() == want.tobytes(), f"call {i}"


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 8, 11, 16])
def test_spmmv_columns_bitwise_equal_spmv(k):
    import torch
    from paper_1307_6209_gb300 import sell

    A = synth.lognormal(3001, seed=6, cap=120)
    X = synth.block(A.ncols, k, seed=5)
    h = sell.sell_build(A, C=32, sigma=128)
    for ld_pad in (0, 3):
        Xd = torch.zeros((A.ncols, k + ld_pad), dtype=torch.float64, device="cuda")
        Xd[:, :k] = torch.from_numpy(X).cuda()
        Yd = torch.full((A.nrows, k + ld_pad), float("nan"), dtype=torch.float64, device="cuda")
        sell.sell_spmmv(h, Xd[:, :k], Yd[:, :k])
        torch.cuda.synchronize()
        Y = Yd[:, :k].cpu().numpy()
        Yref = oracle.csr_spmmv(A, X)
        for c in range(k):
            yc = _spmv(h, X[:, c])
            assert Y[:, c].tobytes() == yc.tobytes(), f"column {c} differs from SpMV"
            scale = oracle.csr_absdot(A, X[:, c])
            assert np.all(np.abs(Y[:, c] - Yref[:, c]) <= tol_f64(A.row_lengths(), scale))
        if ld_pad:
            assert torch.isnan(Yd[:, k:]).all(), "wrote outside the k columns"


def test_spmv_empty_matrix_is_noop():
    import torch
    from paper_1307_6209_gb300 import sell

    A = synth.CSR(0, 0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    h = sell.sell_build(A, C=32, sigma=1)
    sell.sell_spmv(h, torch.empty(0, dtype=torch.float64, device="cuda"),
                   torch.empty(0, dtype=torch.float64, device="cuda"))
    assert h.info.stored == 0 and h.info.nchunks == 0


@pytest.mark.parametrize("shape", ["dense", "one_long_row", "many_long_rows"])
def test_spmv_very_long_rows(shape):
    """Rows of hundreds of 64-entry segments (folded in batches plus a
    remainder) against the oracle, bitwise invariant over (C, sigma)."""
    from paper_1307_6209_gb300 import sell
    if shape == "dense":
        A = synth.dense(300, 2500, seed=1)            # 40 segments per row
    elif shape == "one_long_row":
        A = synth.long_row(30000, 30000, short_len=3, at=777, seed=2)  # 469 segments
    else:
        A = synth.lognormal(3000, mean=900.0, sigma_ln=0.5, cap=3000, seed=3)
    x = synth.vector(A.ncols, seed=4)
    ref, scale, rl = oracle_reference(A, x)
    first = None
    for C, sigma in [(32, 1), (64, 10 ** 9), (7, 100)]:
        h = sell.sell_build(A, C=C, sigma=sigma)
        y = _spmv(h, x)
        assert np.all(np.abs(y - ref) <= tol_f64(rl, scale)), (C, sigma)
        first = y if first is None else first
        assert y.tobytes() == first.tobytes()
        h.free()


@pytest.mark.parametrize("name,A", [
    ("lognormal", synth.lognormal(20011, seed=8, cap=3000)),
    ("empty_and_long", synth.long_row(5000, 5000, short_len=0, at=100, seed=9)),
    ("dense", synth.dense(200, 3000, seed=3)),
    ("random_empty_rows", synth.random_csr(3001, 800, density=0.02, seed=2, empty_rows=0.5)),
], ids=lambda v: v if isinstance(v, str) else "")
def test_bulk_staged_bitwise_equal(name, A):
    """Launch mode 2 (bulk copies into shared memory) gives the bits of mode 0
    for y = A x, y += A x and the single-column block of a wider product
    (strided x and y), for every C it supports, with long rows, chunks of
    empty rows and chunks of long rows only."""
    import torch
    from paper_1307_6209_gb300 import sell

    x = synth.vector(A.ncols, seed=11)
    y0 = synth.vector(A.nrows, seed=12)
    X = synth.block(A.ncols, 5, seed=13)
    for C, sigma in [(32, 1), (32, 10 ** 9), (64, 512), (128, 1)]:
        h = sell.sell_build(A, C=C, sigma=sigma)
        outs = {}
        for mode in (0, 2):
            sell.sell_set_launch(h, 256, 4, mode)
            y = _spmv(h, x)
            ya = _spmv(h, x, y0=y0, flags=sell.SELL_SPMV_ACCUMULATE)
            Xd = torch.from_numpy(X).cuda()
            Yd = torch.full((A.nrows, 5), float("nan"), dtype=torch.float64, device="cuda")
            sell.sell_spmmv(h, Xd, Yd)
            sell.sell_check(h)
            outs[mode] = (y.tobytes(), ya.tobytes(), Yd.cpu().numpy().tobytes())
        assert outs[0] == outs[2], (C, sigma)
        ref, scale, rl = oracle_reference(A, x)
        assert np.all(np.abs(np.frombuffer(outs[2][0]) - ref) <= tol_f64(rl, scale))
        h.free()


def test_spmv_in_cuda_graph():
    """sell_spmv captured in a CUDA graph (long rows included: their counters
    reset themselves, so replays need no clearing) gives the eager bits on
    every replay."""
    import torch
    from paper_1307_6209_gb300 import sell

    A = synth.lognormal(20000, seed=12, cap=3000)
    h = sell.sell_build(A, C=32, sigma=10 ** 9)
    x = torch.from_numpy(synth.vector(A.ncols, seed=2)).cuda()
    y_eager = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
    sell.sell_spmv(h, x, y_eager)  # also sizes the long-row scratch before the capture
    torch.cuda.synchronize()
    y = torch.full((A.nrows,), float("nan"), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for _ in range(3):
            sell.sell_spmv(h, x, y, stream=s)
    for _ in range(4):
        y.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert y.cpu().numpy().tobytes() == y_eager.cpu().numpy().tobytes()


@pytest.mark.parametrize("k", [3, 8, 13])
def test_spmmv_rhs_block_flags_keep_the_bits(k):
    """SELL_SPMV_RHS_BLOCK4/2/1 only narrow the kernel's blocks of
    right-hand sides: the result is the same bits as the default split."""
    import torch
    from paper_1307_6209_gb300 import sell

    A = synth.lognormal(9000, seed=40 + k, cap=1500)
    h = sell.sell_build(A, C=64, sigma=512)
    X = torch.from_numpy(synth.block(A.ncols, k, seed=k)).cuda()
    ref = torch.empty((A.nrows, k), dtype=torch.float64, device="cuda")
    sell.sell_spmmv(h, X, ref)
    for fl in (sell.SELL_SPMV_RHS_BLOCK4, sell.SELL_SPMV_RHS_BLOCK2, sell.SELL_SPMV_RHS_BLOCK1,
               sell.SELL_SPMV_RHS_BLOCK4 | sell.SELL_SPMV_RHS_BLOCK1):
        Y = torch.full((A.nrows, k), float("nan"), dtype=torch.float64, device="cuda")
        sell.sell_spmmv(h, X, Y, flags=fl)
        torch.cuda.synchronize()
        assert torch.equal(Y, ref), f"flags {fl:#x}"


@pytest.mark.parametrize("store,k", [("f64", 4), ("f64", 8), ("f32", 8), ("f32", 16)])
def test_spmmv_row_vector_widths_keep_the_bits(store, k):
    """A row of X is loaded, and a row of Y stored (and read back for
    accumulation), 32 bytes at a time when the base and the pitch are 32-byte
    aligned, 16 bytes at a time when they are 16-byte aligned, value by value
    otherwise.  Pitches k, k + 16 / size and k + 1 and a 16-byte shifted base
    pick each width for X and Y independently; every result is the same bits,
    within the oracle's bound, with and without accumulation, through the
    batch plan as well; Y's padding columns stay untouched."""
    import torch
    from paper_1307_6209_gb300 import sell
    from tests.gpu_util import assert_oracle_parity

    st = {"f64": sell.SELL_F64, "f32": sell.SELL_F32}[store]
    dt = torch.float64 if store == "f64" else torch.float32
    es = 8 if store == "f64" else 4
    A = synth.lognormal(7000, seed=60 + k, cap=900)
    h = sell.sell_build(A, C=64, sigma=4096, store_type=st)
    X0 = torch.from_numpy(synth.block(A.ncols, k, seed=k)).to(dt)
    Y0 = torch.from_numpy(synth.block(A.nrows, k, seed=k + 100)).to(dt)
    layouts = ((k, 0), (k + 16 // es, 0), (k + 1, 0), (k, 16 // es))

    def view(n, ld, shift, fill):
        buf = torch.full((n * ld + shift + 64,), fill, dtype=dt, device="cuda")
        return buf, buf[shift:shift + n * ld].view(n, ld)[:, :k]

    ref = {}
    for acc in (0, sell.SELL_SPMV_ACCUMULATE):
        for (ldx, sx), (ldy, sy) in zip(layouts, layouts[1:] + layouts[:1]):
            _, X = view(A.ncols, ldx, sx, float("nan"))
            X.copy_(X0)
            for batch in (False, True):
                ybuf, Y = view(A.nrows, ldy, sy, -7.0)
                if acc:
                    Y.copy_(Y0)
                else:
                    Y.fill_(float("nan"))
                if batch:
                    plan = sell.sell_batch_create([(h, X, Y, acc)])
                    plan.run()
                    torch.cuda.synchronize()
                    plan.free()
                else:
                    sell.sell_spmmv(h, X, Y, flags=acc)
                    torch.cuda.synchronize()
                if acc not in ref:
                    ref[acc] = Y.clone()
                    assert_oracle_parity(A, st, X0.numpy(), Y.cpu().numpy(), flags=acc,
                                         Y0=Y0.numpy() if acc else None, what=f"{store} k={k} acc={acc}")
                what = f"acc {acc}, ldx {ldx}+{sx}, ldy {ldy}+{sy}, batch {batch}"
                assert torch.equal(Y, ref[acc]), what
                pad = ybuf[sy:sy + A.nrows * ldy].view(A.nrows, ldy)[:, k:]
                assert bool((pad == -7.0).all()), what + ": padding columns written"


@pytest.mark.parametrize("store,comp", [("f64", 0), ("f32", 0), ("f32", 2), ("bf16", 1)])
@pytest.mark.parametrize("k", [4, 8, 12])
def test_spmmv_launch_modes_keep_the_bits(store, comp, k):
    """Launch modes 0 (per-thread loads) and 1 (software-pipelined, at every
    block width of right-hand sides) and every unroll multiply k right-hand
    sides to the same bits, on a matrix with long rows (the segment path) and
    one without; the first result is checked against the oracle."""
    import torch
    from paper_1307_6209_gb300 import sell
    from tests.gpu_util import assert_oracle_parity

    st = {"f64": sell.SELL_F64, "f32": sell.SELL_F32, "bf16": sell.SELL_BF16}[store]
    fl = [0, sell.SELL_SPMV_COMPENSATED, sell.SELL_SPMV_COMPENSATED_LONG][comp]
    dt = torch.float64 if store == "f64" else torch.float32
    for A in (synth.lognormal(6000, seed=70 + k, cap=1500), synth.banded(7000, seed=71 + k)):
        h = sell.sell_build(A, C=64, sigma=512, store_type=st)
        X0 = torch.from_numpy(synth.block(A.ncols, k, seed=k)).to(dt)
        X = X0.cuda()
        ref = None
        for block, unroll, mode in ((128, 1, 0), (128, 2, 1), (256, 4, 1), (128, 1, 1), (512, 8, 1), (128, 4, 0)):
            sell.sell_set_launch(h, block, unroll, mode)
            Y = torch.full((A.nrows, k), float("nan"), dtype=dt, device="cuda")
            sell.sell_spmmv(h, X, Y, flags=fl)
            torch.cuda.synchronize()
            if ref is None:
                ref = Y.clone()
                assert_oracle_parity(A, st, X0.numpy(), Y.cpu().numpy(), flags=fl, what=f"{store} k={k}")
            assert torch.equal(Y, ref), f"block {block} unroll {unroll} mode {mode}"
