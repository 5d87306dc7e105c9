"""Batched products against the oracle.

Every product of a batch plan is checked against the oracle's binary64 CRS
product (Listing "crs") on the stored values, within the bound of the
arithmetic it ran (tests/gpu_util.assert_oracle_parity), and bit for bit
against the same product run alone by sell_spmmv:

* more than 160 products of one kernel variant, so the plan splits the
  variant over several launches (160 products per launch), eagerly and under
  a captured CUDA graph;
* a mixed set of every variant (binary64 / binary32 / bfloat16 storage,
  plain and compensated accumulation, 1-16 right-hand sides, accumulate);
* the benchmark's 512-matrix batch itself (rows U[1000, 200000], half banded,
  half lognormal, binary32), at 1 and 8 right-hand sides.
"""
import numpy as np
import pytest

from paper_1307_6209_gb300 import synth
from tests.gpu_util import assert_oracle_parity, host_csr

pytestmark = pytest.mark.gpu


def _alone(h, X, Y0, fl):
    import torch
    from paper_1307_6209_gb300 import sell
    if Y0 is not None:
        Y = Y0.clone()
    else:
        shape = (h.info.nrows,) if X.dim() == 1 else (h.info.nrows, X.shape[1])
        Y = torch.full(shape, float("nan"), dtype=X.dtype, device="cuda")
    if X.dim() == 1:
        sell.sell_spmv(h, X, Y, flags=fl)
    else:
        sell.sell_spmmv(h, X, Y, flags=fl)
    return Y


def _product(A, store, k, fl, seed, C, sigma, acc=False):
    """(handle, host CSR, X, Y, Y0 or None, flags) for one batch item."""
    import torch
    from paper_1307_6209_gb300 import sell
    h = sell.sell_build(A, C=C, sigma=sigma, store_type=store)
    dt = torch.float64 if store == sell.SELL_F64 else torch.float32
    X = torch.from_numpy(synth.block(A.ncols, k, seed=seed)).to(dt)
    if k == 1:
        X = X[:, 0].contiguous()
    X = X.cuda()
    shape = (A.nrows,) if k == 1 else (A.nrows, k)
    Y0 = None
    if acc:
        fl |= sell.SELL_SPMV_ACCUMULATE
        Y0 = torch.from_numpy(synth.block(A.nrows, k, seed=seed + 1)).to(dt).reshape(shape).cuda()
        Y = Y0.clone()
    else:
        Y = torch.full(shape, float("nan"), dtype=dt, device="cuda")
    return h, A, X, Y, Y0, fl


def _check(prods, what):
    """Each product's Y against the oracle and against the product alone."""
    for i, (h, A, X, Y, Y0, fl) in enumerate(prods):
        got = Y.cpu().numpy()
        assert_oracle_parity(A, h.info.store_type, X.cpu().numpy(), got, flags=fl,
                             Y0=None if Y0 is None else Y0.cpu().numpy(), what=f"{what} product {i}")
        ya = _alone(h, X, Y0, fl)
        assert got.tobytes() == ya.cpu().numpy().tobytes(), f"{what} product {i}: batch != alone"


def _one_variant_set(n=200):
    """n small binary32 products of one right-hand side and plain accumulation
    (a single kernel variant), over banded, lognormal, empty-row and long-row
    matrices; two products share each of the first matrices."""
    rng = np.random.default_rng(11)
    fmts = [(32, 1), (32, 256), (64, 4096), (128, 10 ** 9)]
    prods, mats = [], []
    for i in range(n):
        if i < 20 and i % 2 == 1:
            A = mats[-1]  # the same matrix as the previous product, another x
        else:
            N = int(rng.integers(40, 2500))
            kind = i % 4
            if kind == 0:
                A = synth.banded(N, seed=i)
            elif kind == 1:
                A = synth.lognormal(N, seed=i, cap=400)
            elif kind == 2:
                A = synth.random_csr(N, N, density=0.01, seed=i, empty_rows=0.3)
            else:
                A = synth.long_row(N, min(N, 1500), short_len=3, at=N // 2, seed=i)
            mats.append(A)
        C, sigma = fmts[i % 4]
        prods.append(_product(A, 1, 1, 0, seed=1000 + i, C=C, sigma=sigma, acc=(i % 7 == 3)))
    return prods


def test_batch_one_variant_split_over_launches():
    import torch
    from paper_1307_6209_gb300 import sell

    prods = _one_variant_set(200)  # > 160 products of one variant: two launches
    items = [(h, X, Y, fl) for h, A, X, Y, Y0, fl in prods]
    plan = sell.sell_batch_create(items)
    plan.run()
    torch.cuda.synchronize()
    _check(prods, "eager")
    # the same plan captured in a CUDA graph and replayed
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(stream=s)
    for h, A, X, Y, Y0, fl in prods:
        if Y0 is not None:
            Y.copy_(Y0)
        else:
            Y.fill_(float("nan"))
    with torch.cuda.stream(s):
        g.replay()
    torch.cuda.synchronize()
    _check(prods, "graph")
    plan.free()


def test_batch_every_variant_vs_oracle():
    import torch
    from paper_1307_6209_gb300 import sell

    rng = np.random.default_rng(12)
    prods = []
    i = 0
    for store in (sell.SELL_F64, sell.SELL_F32, sell.SELL_BF16):
        comps = [0] if store == sell.SELL_F64 else [0, sell.SELL_SPMV_COMPENSATED, sell.SELL_SPMV_COMPENSATED_LONG]
        for fl in comps:
            for k in (1, 2, 3, 4, 5, 8, 9, 16):
                N = int(rng.integers(100, 6000))
                A = synth.lognormal(N, seed=200 + i, cap=1200) if i % 2 else synth.banded(N, seed=200 + i)
                C, sigma = [(32, 1), (64, 512), (128, 10 ** 9)][i % 3]
                prods.append(_product(A, store, k, fl, seed=3000 + i, C=C, sigma=sigma, acc=(i % 5 == 2)))
                i += 1
    plan = sell.sell_batch_create([(h, X, Y, fl) for h, A, X, Y, Y0, fl in prods])
    plan.run()
    torch.cuda.synchronize()
    _check(prods, "mixed")
    plan.free()


@pytest.mark.parametrize("k", [1, 8])
def test_batch_benchmark_set(k):
    """The 512-matrix binary32 batch of the benchmark: every product bitwise
    equal to the product alone, and a sample of 24 products (both kinds, the
    largest and the smallest among them) against the oracle."""
    import torch
    from paper_1307_6209_gb300 import sell

    recipe = synth.batch_set(512, seed=0)
    gen = {"banded": synth.banded_device, "lognormal": synth.lognormal_device}
    rng = np.random.default_rng(13)
    order = np.argsort([n for _, n, _ in recipe])
    sample = set(rng.choice(512, 20, replace=False).tolist()) | {int(order[0]), int(order[1]),
                                                                  int(order[-1]), int(order[-2])}
    hs, host = [], {}
    for i, (kind, n, seed) in enumerate(recipe):
        A = gen[kind](n, seed=seed)
        C, sigma = (32, 1) if kind == "banded" else (32, n)  # the results do not depend on C and sigma
        hs.append(sell.sell_build(A, C=C, sigma=sigma, store_type=sell.SELL_F32))
        if i in sample:
            host[i] = host_csr(A)
        del A
    items = []
    for i, h in enumerate(hs):
        shp_x = (h.info.ncols,) if k == 1 else (h.info.ncols, k)
        shp_y = (h.info.nrows,) if k == 1 else (h.info.nrows, k)
        g = torch.Generator(device="cuda").manual_seed(i)
        X = torch.rand(shp_x, dtype=torch.float32, device="cuda", generator=g) * 2 - 1
        items.append((h, X, torch.full(shp_y, float("nan"), dtype=torch.float32, device="cuda"), 0))
    plan = sell.sell_batch_create(items)
    plan.run()
    torch.cuda.synchronize()
    for i, (h, X, Y, fl) in enumerate(items):
        ya = _alone(h, X, None, 0)
        assert torch.equal(Y, ya), f"product {i}: batch != alone"
        if i in host:
            assert_oracle_parity(host[i], sell.SELL_F32, X.cpu().numpy(), Y.cpu().numpy(), what=f"product {i}")
    plan.free()
    for h in hs:
        h.free()


def test_batch_tuning_knobs_keep_the_bits():
    """The autotuner's knobs of a batch -- the right-hand-side block width of
    each item (SELL_SPMV_RHS_BLOCK4/2/1) and the plan's block size (64, 128,
    256 rows per work unit) -- change no bit of any product."""
    import torch
    from paper_1307_6209_gb300 import sell

    rng = np.random.default_rng(14)
    prods = []
    for i in range(12):
        N = int(rng.integers(300, 5000))
        A = synth.lognormal(N, seed=400 + i, cap=900) if i % 2 else synth.banded(N, seed=400 + i)
        store = [sell.SELL_F64, sell.SELL_F32, sell.SELL_BF16][i % 3]
        prods.append(_product(A, store, [8, 5, 16][i % 3], 0, seed=500 + i, C=32, sigma=[1, 256][i % 2]))
    plan = sell.sell_batch_create([(h, X, Y, fl) for h, A, X, Y, Y0, fl in prods])
    plan.run()
    torch.cuda.synchronize()
    ref = [Y.clone() for _, _, _, Y, _, _ in prods]
    _check(prods, "default")
    plan.free()
    for rhs in (sell.SELL_SPMV_RHS_BLOCK4, sell.SELL_SPMV_RHS_BLOCK2, sell.SELL_SPMV_RHS_BLOCK1):
        for block in (64, 128, 256):
            for _, _, _, Y, _, _ in prods:
                Y.fill_(float("nan"))
            plan = sell.sell_batch_create([(h, X, Y, fl | rhs) for h, A, X, Y, Y0, fl in prods])
            plan.set_launch(block)
            plan.run()
            torch.cuda.synchronize()
            for (h, A, X, Y, Y0, fl), r in zip(prods, ref):
                assert torch.equal(Y, r), f"rhs flag {rhs:#x}, block {block}"
            plan.free()
    plan = sell.sell_batch_create([(h, X, Y, fl) for h, A, X, Y, Y0, fl in prods])
    with pytest.raises(sell.SellError) as e:
        plan.set_launch(96)
    assert e.value.status == sell.SELL_EINVAL
    plan.free()
