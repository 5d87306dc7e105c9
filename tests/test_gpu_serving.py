"""Continuous-batching server: every result equals the same request run alone
(bitwise), requests that arrive while others run are admitted and overlap,
and the HBM budget is never exceeded."""
import threading
import time

import numpy as np
import pytest

from paper_1307_6209_gb300 import synth

pytestmark = pytest.mark.gpu


def _mats(seed=0):
    from paper_1307_6209_gb300 import sell
    mats = []
    for i, n in enumerate([3000, 50000, 20000, 120000, 7000, 60000]):
        A = synth.lognormal_device(n, seed=seed + i, cap=800)
        st = sell.SELL_F64 if i % 2 == 0 else sell.SELL_F32
        mats.append(sell.sell_build(A, C=32, sigma=n if i % 3 else 1, store_type=st))
    return mats


def _make(mats, rng):
    import torch
    from paper_1307_6209_gb300 import sell
    mid = int(rng.integers(0, len(mats)))
    inf = mats[mid].info
    k = int(rng.integers(1, 9))
    dt = torch.float64 if inf.store_type == sell.SELL_F64 else torch.float32
    X = torch.from_numpy(rng.uniform(-1, 1, (inf.ncols, k))).to(dt)
    if k == 1 and rng.random() < 0.5:
        X = X[:, 0].contiguous()
    return mid, X.pin_memory()


def _alone(h, X):
    import torch
    from paper_1307_6209_gb300 import sell
    Xd = X.cuda()
    if X.dim() == 1:
        Y = torch.empty(h.info.nrows, dtype=X.dtype, device="cuda")
        sell.sell_spmv(h, Xd, Y)
    else:
        Y = torch.empty((h.info.nrows, X.shape[1]), dtype=X.dtype, device="cuda")
        sell.sell_spmmv(h, Xd, Y)
    torch.cuda.synchronize()
    return Y.cpu()


def test_results_alone_equal_in_the_mix():
    from paper_1307_6209_gb300 import serving
    mats = _mats()
    srv = serving.Server(mats, hbm_budget_bytes=8 << 30, max_batch=16, streams=3).start()
    rng = np.random.default_rng(1)
    reqs = []
    # bursts: many requests arrive while earlier batches are on the GPU
    for burst in range(6):
        for _ in range(int(rng.integers(5, 30))):
            mid, X = _make(mats, rng)
            reqs.append(srv.submit(mid, X, to_host=bool(rng.random() < 0.7)))
        time.sleep(0.002)
    for r in reqs:
        assert r.done.wait(60)
    srv.stop()
    st = srv.stats()
    assert st["requests"] == len(reqs) and st["batches"] >= 2
    for r in reqs:
        ref = _alone(mats[r.mid], r.X)
        got = r.Y.cpu() if r.Y.is_cuda else r.Y
        assert got.numpy().tobytes() == ref.numpy().tobytes(), f"request {r.rid} differs"


def test_budget_is_respected_and_everything_completes():
    from paper_1307_6209_gb300 import serving
    mats = _mats(seed=10)
    resident = sum(h.info.device_bytes for h in mats)
    srv_probe = serving.Server(mats, hbm_budget_bytes=resident + (1 << 30))
    biggest = max(srv_probe.request_bytes(i, 8) for i in range(len(mats)))
    budget = resident + biggest  # room for about one large request at a time
    srv = serving.Server(mats, hbm_budget_bytes=budget, max_batch=64, streams=3).start()
    rng = np.random.default_rng(2)
    reqs = [srv.submit(*_make(mats, rng)) for _ in range(60)]
    for r in reqs:
        assert r.done.wait(60)
    srv.stop()
    st = srv.stats()
    assert st["peak_hbm_bytes"] <= budget
    assert st["requests"] == 60
    with pytest.raises(ValueError):
        serving.Server(mats, hbm_budget_bytes=resident - 1)
    small = serving.Server(mats, hbm_budget_bytes=resident + 16)
    import torch
    with pytest.raises(ValueError):
        small.submit(1, torch.zeros(mats[1].info.ncols, dtype=torch.float32))


def test_poisson_load_reports_latency():
    from paper_1307_6209_gb300 import serving
    mats = _mats(seed=20)
    srv = serving.Server(mats, hbm_budget_bytes=8 << 30, streams=3).start()
    reqs = serving.poisson_load(srv, rate_hz=2000.0, duration_s=0.3, make_request=lambda g: _make(mats, g))
    for r in reqs:
        assert r.done.wait(60)
    srv.stop()
    st = srv.stats()
    assert st["requests"] == len(reqs) > 100
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    assert all(r.t_arrive <= r.t_launch <= r.t_done for r in reqs)
