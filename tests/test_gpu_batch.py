"""Batched persistent launches: every product of a batch is bitwise equal to
the same product run alone (the per-row operation order does not depend on
the batch), for mixed sizes, storage types and right-hand-side counts."""
import numpy as np
import pytest

from paper_1307_6209_gb300 import synth

pytestmark = pytest.mark.gpu


def _make_products(seed=0, n=24):
    import torch
    from paper_1307_6209_gb300 import sell

    rng = np.random.default_rng(seed)
    prods = []
    for i in range(n):
        N = int(rng.integers(50, 20000))
        A = synth.banded(N, seed=i) if i % 2 else synth.lognormal(N, seed=i, cap=300)
        store = [sell.SELL_F64, sell.SELL_F32, sell.SELL_BF16][i % 3]
        k = [1, 2, 3, 4, 8, 9][i % 6]
        C, sigma = [(32, 1), (32, 256), (64, 4096), (128, 10 ** 9)][i % 4]
        h = sell.sell_build(A, C=C, sigma=sigma, store_type=store)
        dt = torch.float64 if store == sell.SELL_F64 else torch.float32
        X = torch.from_numpy(synth.block(A.ncols, k, seed=100 + i)).to(dt).cuda()
        Y = torch.full((A.nrows, k), float("nan"), dtype=dt, device="cuda")
        fl = 0
        if store != sell.SELL_F64 and i % 4 == 1:
            fl = sell.SELL_SPMV_COMPENSATED
        elif store != sell.SELL_F64 and i % 4 == 3:
            fl = sell.SELL_SPMV_COMPENSATED_LONG
        prods.append((h, X, Y, fl))
    return prods


def test_batch_equals_alone():
    import torch
    from paper_1307_6209_gb300 import sell

    prods = _make_products()
    alone = []
    for h, X, Y, fl in prods:
        Ya = torch.empty_like(Y)
        sell.sell_spmmv(h, X, Ya, flags=fl)
        alone.append(Ya)
    plan = sell.sell_batch_create(prods)
    for rep in range(3):
        for _, _, Y, _ in prods:
            Y.fill_(float("nan"))
        plan.run()
        torch.cuda.synchronize()
        for (h, X, Y, fl), Ya in zip(prods, alone):
            assert Y.cpu().numpy().tobytes() == Ya.cpu().numpy().tobytes()
    plan.free()


def test_batch_in_cuda_graph():
    import torch
    from paper_1307_6209_gb300 import sell

    prods = _make_products(seed=1, n=10)
    plan = sell.sell_batch_create(prods)
    s = torch.cuda.Stream()
    plan.run(stream=s)  # warm-up outside capture
    torch.cuda.synchronize()
    ref = [Y.clone() for _, _, Y, _ in prods]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(stream=s)
    for _, _, Y, _ in prods:
        Y.fill_(float("nan"))
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    for (_, _, Y, _), r in zip(prods, ref):
        assert torch.equal(Y, r)


def test_batch_empty_and_bad_items():
    from paper_1307_6209_gb300 import sell
    plan = sell.sell_batch_create([])
    plan.run()
    plan.free()
    prods = _make_products(seed=3, n=2)
    plan = sell.sell_batch_create(prods)
    with pytest.raises(sell.SellError) as e:
        plan.run(grid=5)
    assert e.value.status == sell.SELL_EINVAL
    plan.free()
