"""Continuous-batching server: every result equals the same request run alone
(bitwise) and agrees with the oracle's binary64 CRS product within the bound
of its storage type, requests that arrive while others run are admitted and
overlap, and the HBM budget is never exceeded."""
import threading
import time

import numpy as np
import pytest

from paper_1307_6209_gb300 import synth
from tests.gpu_util import assert_oracle_parity, host_csr

pytestmark = pytest.mark.gpu


def _mats(seed=0, hosts=None):
    """Six resident matrices (binary64 and binary32 storage); with `hosts`, a
    host copy of each CSR is appended for the oracle."""
    from paper_1307_6209_gb300 import sell
    mats = []
    for i, n in enumerate([3000, 50000, 20000, 120000, 7000, 60000]):
        A = synth.lognormal_device(n, seed=seed + i, cap=800)
        st = sell.SELL_F64 if i % 2 == 0 else sell.SELL_F32
        mats.append(sell.sell_build(A, C=32, sigma=n if i % 3 else 1, store_type=st))
        if hosts is not None:
            hosts.append(host_csr(A))
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
    hosts = []
    mats = _mats(hosts=hosts)
    srv = serving.Server(mats, hbm_budget_bytes=8 << 30, max_batch=16, streams=3).start()
    rng = np.random.default_rng(1)
    reqs = []
    # bursts: many requests arrive while earlier batches are on the GPU
    for burst in range(6):
        for _ in range(int(rng.integers(5, 30))):
            mid, X = _make(mats, rng)
            reqs.append(srv.submit(mid, X, to_host=bool(rng.random() < 0.7)))
        time.sleep(0.002)
    got = []
    for r in reqs:
        r.wait(60)
        got.append(r.result().cpu().clone())
        r.release()
    st = srv.stats()
    srv.stop()
    assert st["requests"] == len(reqs) and st["batches"] >= 2
    ks = set()
    for r, y in zip(reqs, got):
        ref = _alone(mats[r.mid], r.X)
        assert y.numpy().tobytes() == ref.numpy().tobytes(), f"request {r.rid} differs"
        assert_oracle_parity(hosts[r.mid], mats[r.mid].info.store_type, r.X.numpy(), y.numpy(),
                             what=f"request {r.rid}")
        ks.add((mats[r.mid].info.store_type, 1 if r.X.dim() == 1 else r.X.shape[1]))
    assert {st for st, _ in ks} == {0, 1} and max(k for _, k in ks) >= 6


def test_requests_arriving_during_a_batch_share_the_next_launch():
    """With one stream, requests queued while a long product runs are admitted
    together into the next launch, and every result still equals the request
    alone."""
    import torch
    from paper_1307_6209_gb300 import serving, sell
    Abig = synth.lognormal_device(2_000_000, seed=5)
    big = sell.sell_build(Abig, C=32, sigma=2_000_000)
    hosts = []
    mats = _mats(seed=40, hosts=hosts) + [big]
    hosts.append(host_csr(Abig))
    del Abig
    srv = serving.Server(mats, hbm_budget_bytes=sum(m.info.device_bytes for m in mats) + (4 << 30),
                         max_batch=64, streams=1)
    Xb = torch.rand((big.info.ncols, 8), dtype=torch.float64).pin_memory()
    rng = np.random.default_rng(6)
    made = [_make(mats[:-1], rng) for _ in range(10)]  # inputs ready before the first submit
    first = srv.submit(len(mats) - 1, Xb, to_host=False)
    rest = [srv.submit(mid, X, to_host=True) for mid, X in made]
    for r in [first] + rest:
        r.wait(60)
    ybig = first.result().cpu().clone()
    first.release()
    srv.stop()
    assert max(r.batch for r in rest) > 1, "queued requests did not share a launch"
    assert all(r.t_launch >= first.t_launch for r in rest)
    assert ybig.numpy().tobytes() == _alone(big, Xb).numpy().tobytes()
    assert_oracle_parity(hosts[-1], sell.SELL_F64, Xb.numpy(), ybig.numpy(), what="2M-row request")
    for r in rest:
        assert r.Y.numpy().tobytes() == _alone(mats[r.mid], r.X).numpy().tobytes()
        assert_oracle_parity(hosts[r.mid], mats[r.mid].info.store_type, r.X.numpy(), r.Y.numpy(),
                             what=f"request {r.rid}")


def test_budget_is_respected_and_everything_completes():
    from paper_1307_6209_gb300 import serving
    mats = _mats(seed=10)
    resident = sum(h.info.device_bytes for h in mats)
    biggest = max((mats[i].info.ncols + mats[i].info.nrows) * 8 * 8 for i in range(len(mats)))
    budget = resident + 2 * biggest  # room for about one large request at a time (plus scratch)
    srv = serving.Server(mats, hbm_budget_bytes=budget, max_batch=64, streams=3).start()
    rng = np.random.default_rng(2)
    reqs = [srv.submit(*_make(mats, rng)) for _ in range(60)]
    for r in reqs:
        r.wait(60)
    st = srv.stats()
    srv.stop()
    assert st["peak_hbm_bytes"] <= budget
    assert st["requests"] == 60
    with pytest.raises(ValueError):
        serving.Server(mats, hbm_budget_bytes=resident)
    small = serving.Server(mats, hbm_budget_bytes=resident + 4096)
    import torch
    with pytest.raises(ValueError):
        small.submit(1, torch.zeros(mats[1].info.ncols, dtype=torch.float32).pin_memory())
    with pytest.raises(ValueError):  # pageable host memory is refused
        small.submit(0, torch.zeros(4, dtype=torch.float64))
    small.stop()


def test_poisson_load_reports_latency():
    from paper_1307_6209_gb300 import serving
    mats = _mats(seed=20)
    srv = serving.Server(mats, hbm_budget_bytes=8 << 30, streams=3).start()
    reqs = serving.poisson_load(srv, rate_hz=2000.0, duration_s=0.3, make_request=lambda g: _make(mats, g),
                                to_host=False)
    st = srv.stats()
    srv.stop()
    assert st["requests"] == len(reqs) > 100
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    assert all(r.t_arrive <= r.t_launch <= r.t_done for r in reqs)


def test_native_accumulate_and_errors():
    """Y += A X through the C entry points with a host y; unknown ids and
    waits that time out are reported, not hung on."""
    import torch
    from paper_1307_6209_gb300 import sell
    mats = _mats(seed=30)
    h = mats[2]
    srv = sell.sell_server_create(mats, sum(m.info.device_bytes for m in mats) + (1 << 30), 8, 2)
    try:
        x = torch.from_numpy(synth.vector(h.info.ncols, seed=3)).pin_memory()
        y0 = synth.vector(h.info.nrows, seed=4)
        y = torch.from_numpy(y0.copy()).pin_memory()
        rid = sell.sell_server_submit(srv, 2, x.data_ptr(), 1, y.data_ptr(), sell.SELL_SPMV_ACCUMULATE)
        info = sell.sell_server_wait(srv, rid, 60.0)
        assert info.status == sell.SELL_OK and info.t_done >= info.t_launch >= info.t_arrive
        yd = torch.from_numpy(y0.copy()).cuda()
        sell.sell_spmv(h, x.cuda(), yd, flags=sell.SELL_SPMV_ACCUMULATE)
        torch.cuda.synchronize()
        assert y.numpy().tobytes() == yd.cpu().numpy().tobytes()
        with pytest.raises(sell.SellError) as e:
            sell.sell_server_wait(srv, rid, 1.0)  # a host-result request is forgotten after its wait
        assert e.value.status == sell.SELL_EINVAL
        # completion-order delivery: two device results, each delivered once
        x1 = torch.ones(mats[1].info.ncols, dtype=torch.float32).pin_memory()
        x3 = torch.ones(mats[3].info.ncols, dtype=torch.float32).pin_memory()
        r1 = sell.sell_server_submit(srv, 1, x1.data_ptr(), 1, None)
        r2 = sell.sell_server_submit(srv, 3, x3.data_ptr(), 1, None)
        got = {sell.sell_server_next(srv, 60.0)[0], sell.sell_server_next(srv, 60.0)[0]}
        assert got == {r1, r2}
        with pytest.raises(sell.SellError) as e:
            sell.sell_server_next(srv, 0.05)
        assert e.value.status == sell.SELL_ETIMEOUT
        for r in (r1, r2):
            assert sell.sell_server_result(srv, r)
            sell.sell_server_release(srv, r)
        with pytest.raises(sell.SellError) as e:  # accumulating needs a host y
            sell.sell_server_submit(srv, 2, x.data_ptr(), 1, None, sell.SELL_SPMV_ACCUMULATE)
        assert e.value.status == sell.SELL_EINVAL
        with pytest.raises(sell.SellError) as e:
            sell.sell_server_submit(srv, 0, x.data_ptr(), 1, None, sell.SELL_SPMV_COMPENSATED)
        assert e.value.status == sell.SELL_EUNSUPPORTED
    finally:
        sell.sell_server_destroy(srv)


def test_destroy_with_unreleased_results_does_not_wait_forever():
    """A device result that is never released blocks a queued request that
    needs its memory; destroying the server drops the held result, lets the
    queued request finish and returns."""
    import torch
    from paper_1307_6209_gb300 import sell
    n = 50000
    h = sell.sell_build(synth.lognormal_device(n, seed=60, cap=64), C=32, sigma=n, store_type=sell.SELL_F32)
    # no long rows, so a k = 2 request needs exactly its x and y blocks: 16 n
    # bytes; the arena holds one request (20 n), and a second one only once
    # the first result's 8 n bytes are released
    srv = sell.sell_server_create([h], h.info.device_bytes + 20 * n, 4, 2)
    x = torch.ones((n, 2), dtype=torch.float32).pin_memory()
    held = sell.sell_server_submit(srv, 0, x.data_ptr(), 2, None)
    sell.sell_server_wait(srv, held, 60.0)
    blocked = sell.sell_server_submit(srv, 0, x.data_ptr(), 2, None)
    time.sleep(0.2)
    st = sell.sell_server_stats(srv)
    assert st["queued"] == 1  # waits for the held result's memory
    done = threading.Event()
    t = threading.Thread(target=lambda: (sell.sell_server_destroy(srv), done.set()), daemon=True)
    t.start()
    t.join(60)
    assert done.is_set(), "sell_server_destroy did not return"
    assert blocked


def test_size_ratio_batches_keep_results_and_order():
    """With a size ratio the oldest request still goes first and every result
    is the request alone; batches then hold requests of similar work."""
    from paper_1307_6209_gb300 import serving
    mats = _mats(seed=70)
    srv = serving.Server(mats, hbm_budget_bytes=8 << 30, max_batch=32, streams=2, size_ratio=4)
    rng = np.random.default_rng(3)
    made = [_make(mats, rng) for _ in range(40)]
    reqs = [srv.submit(mid, X, to_host=True) for mid, X in made]
    for r in reqs:
        r.wait(60)
    srv.stop()
    for r in reqs:
        assert r.Y.numpy().tobytes() == _alone(mats[r.mid], r.X).numpy().tobytes()
    assert reqs[0].t_launch <= min(r.t_launch for r in reqs[1:])


def test_wait_and_next_racing_for_one_request():
    """One thread waits on a request while another takes the next completed
    request: exactly one of the two delivers it, and the other gets an error
    (never a request that was freed while it slept)."""
    import torch
    from paper_1307_6209_gb300 import sell
    A = synth.lognormal_device(20000, seed=3, cap=500)
    h = sell.sell_build(A, C=32, sigma=20000)
    srv = sell.sell_server_create([h], budget_bytes=1 << 30, max_batch=4, streams=1)
    try:
        for _ in range(8):
            X = torch.rand(A.ncols, dtype=torch.float64).pin_memory()
            Y = torch.empty(A.nrows, dtype=torch.float64).pin_memory()
            rid = sell.sell_server_submit(srv, 0, X.data_ptr(), 1, Y.data_ptr())
            out = {}

            def waiter():
                try:
                    sell.sell_server_wait(srv, rid, 10.0)
                    out["wait"] = "ok"
                except sell.SellError as e:
                    out["wait"] = e.status

            t = threading.Thread(target=waiter)
            t.start()
            try:
                out["next"] = sell.sell_server_next(srv, 1.0)[0]
            except sell.SellError as e:
                out["next"] = e.status
            t.join(20)
            assert not t.is_alive()
            if out["wait"] == "ok":
                assert out["next"] == sell.SELL_ETIMEOUT
            else:
                assert out["wait"] == sell.SELL_EINVAL and out["next"] == rid
    finally:
        sell.sell_server_destroy(srv)
        h.free()


def test_small_inputs_are_copied_ahead_of_a_large_one():
    """Input copies on different streams share the copy engine first in,
    first out, so the server meters them: a large request's 128 MB input goes
    in chunks, and the inputs of small requests submitted just after it are
    copied between its chunks -- they complete before it does.  Every result
    is still the request alone, and the oracle's product within its bound."""
    import torch
    from paper_1307_6209_gb300 import serving, sell
    Abig = synth.lognormal_device(2_000_000, seed=16)
    big = sell.sell_build(Abig, C=32, sigma=2_000_000)
    hosts = []
    mats = _mats(seed=90, hosts=hosts) + [big]
    hosts.append(host_csr(Abig))
    del Abig
    srv = serving.Server(mats, hbm_budget_bytes=sum(m.info.device_bytes for m in mats) + (4 << 30), max_batch=8,
                         streams=4)
    Xb = torch.rand((big.info.ncols, 8), dtype=torch.float64).pin_memory()
    rng = np.random.default_rng(10)
    small_x = [torch.rand(mats[0].info.ncols, dtype=torch.float64).pin_memory() for _ in range(6)]
    large = srv.submit(len(mats) - 1, Xb, to_host=True)
    small = [srv.submit(0, x, to_host=True) for x in small_x]
    for r in [large] + small:
        r.wait(60)
    srv.stop()
    assert min(r.t_done for r in small) < large.t_done, "every small request waited for the large input"
    assert large.Y.numpy().tobytes() == _alone(big, Xb).numpy().tobytes()
    assert_oracle_parity(hosts[-1], sell.SELL_F64, Xb.numpy(), large.Y.numpy(), what="large request")
    for r in small:
        assert r.Y.numpy().tobytes() == _alone(mats[0], r.X).numpy().tobytes()
        assert_oracle_parity(hosts[0], mats[0].info.store_type, r.X.numpy(), r.Y.numpy(), what=f"request {r.rid}")


def test_small_requests_of_a_mixed_batch_complete_first():
    """A batch that mixes small and large products runs in two parts on its
    stream, the small products first with their own completion event: small
    requests admitted together with a large one complete before it.  Every
    result is the request alone, and the oracle's product within its bound."""
    import torch
    from paper_1307_6209_gb300 import serving, sell
    Abig = synth.lognormal_device(2_000_000, seed=17)
    big = sell.sell_build(Abig, C=32, sigma=2_000_000)
    hosts = []
    mats = _mats(seed=95, hosts=hosts) + [big]
    hosts.append(host_csr(Abig))
    del Abig
    # one stream: the first large request runs alone; the next ones queue
    # meanwhile and are admitted together as one mixed batch
    srv = serving.Server(mats, hbm_budget_bytes=sum(m.info.device_bytes for m in mats) + (4 << 30), max_batch=16,
                         streams=1)
    Xb = [torch.rand((big.info.ncols, 8), dtype=torch.float64).pin_memory() for _ in range(2)]
    small_x = [torch.rand((mats[0].info.ncols, 2), dtype=torch.float64).pin_memory() for _ in range(4)]
    first = srv.submit(len(mats) - 1, Xb[0], to_host=True)
    large = srv.submit(len(mats) - 1, Xb[1], to_host=True)
    small = [srv.submit(0, x, to_host=True) for x in small_x]
    for r in [first, large] + small:
        r.wait(60)
    srv.stop()
    mixed = [r for r in small if r.t_launch == large.t_launch]
    assert mixed, "no small request shared the large one's batch"
    assert max(r.t_done for r in mixed) < large.t_done, "the small part did not complete first"
    for r in [first, large]:
        assert r.Y.numpy().tobytes() == _alone(big, r.X).numpy().tobytes()
    assert_oracle_parity(hosts[-1], sell.SELL_F64, large.X.numpy(), large.Y.numpy(), what="large request")
    for r in small:
        assert r.Y.numpy().tobytes() == _alone(mats[0], r.X).numpy().tobytes()
        assert_oracle_parity(hosts[0], mats[0].info.store_type, r.X.numpy(), r.Y.numpy(), what=f"request {r.rid}")
