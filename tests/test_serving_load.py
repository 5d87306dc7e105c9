"""The serving benchmark's load generators and client thread, on the CPU.

poisson_load must submit requests with exponential inter-arrival times at
the requested rate and burst_load all at once; the client thread must take
every request in completion order and release it.  A fake server stands in
for the native one (it completes each request as soon as it is submitted),
so only the Python side is under test.  Bounds are loose enough for a busy
host: the count within 5 standard deviations of the Poisson mean, the mean
gap within 10 %, the coefficient of variation of the gaps near 1.
"""
import queue
import time

import numpy as np

from paper_1307_6209_gb300 import sell, serving


class _FakeRequest:
    def __init__(self, mid, X):
        self.mid, self.X, self.released = mid, X, False

    def release(self):
        self.released = True


class _FakeServer:
    def __init__(self):
        self.q = queue.Queue()
        self.t = []

    def submit(self, mid, X, to_host=True):
        r = _FakeRequest(mid, X)
        self.t.append(time.perf_counter())
        self.q.put(r)
        return r

    def next(self, timeout):
        try:
            return self.q.get(timeout=timeout)
        except queue.Empty:
            raise sell.SellError(sell.SELL_ETIMEOUT, "no request completed in time")


def _make(rng):
    return int(rng.integers(0, 4)), None


def test_poisson_arrivals_rate_and_gaps():
    srv = _FakeServer()
    rate, dur = 1000.0, 1.5
    reqs = serving.poisson_load(srv, rate, dur, _make, seed=3)
    n = len(reqs)
    assert abs(n - rate * dur) < 5 * np.sqrt(rate * dur)
    assert all(r.released for r in reqs)  # the client thread took and released every one
    gaps = np.diff(np.array(srv.t))
    assert abs(gaps.mean() - 1.0 / rate) < 0.1 / rate
    cv = gaps.std() / gaps.mean()
    assert 0.8 < cv < 1.2  # exponential gaps: cv = 1 (a fixed-rate stream would give 0)


def test_poisson_arrivals_are_seeded():
    a = serving.poisson_load(_FakeServer(), 2000.0, 0.3, _make, seed=5)
    b = serving.poisson_load(_FakeServer(), 2000.0, 0.3, _make, seed=5)
    assert [r.mid for r in a] == [r.mid for r in b]


def test_burst_load_submits_all_and_collects_all():
    srv = _FakeServer()
    reqs, secs = serving.burst_load(srv, 500, _make, seed=1)
    assert len(reqs) == 500 and all(r.released for r in reqs) and secs >= 0
    assert srv.t[-1] - srv.t[0] < 0.5  # all at once, not paced


class _OneAtATimeServer(_FakeServer):
    """Completes one request per `service` seconds, in submission order,
    on a worker thread; records how many were in the server at once."""

    def __init__(self, service):
        super().__init__()
        import threading
        self.service, self.pending, self.live, self.max_live = service, queue.Queue(), 0, 0
        self.lock = threading.Lock()
        self.submitted = []
        threading.Thread(target=self._work, daemon=True).start()

    def submit(self, mid, X, to_host=True):
        r = _FakeRequest(mid, X)
        with self.lock:
            self.live += 1
            self.max_live = max(self.max_live, self.live)
        self.submitted.append(r)
        self.pending.put(r)
        return r

    def _work(self):
        while True:
            r = self.pending.get()
            time.sleep(self.service)
            with self.lock:
                self.live -= 1
            self.q.put(r)


def test_closed_loop_keeps_the_window_full_and_measures_the_service_rate():
    srv = _OneAtATimeServer(0.002)
    done, secs = serving.closed_loop(srv, 8, 0.5, _make, seed=2)
    assert srv.max_live <= 8  # never more than the window outstanding
    assert all(r.released for r in srv.submitted)  # drained and released
    assert srv.live == 0 and srv.q.empty()
    rate = done / secs
    assert 0.5 / 0.002 < rate <= 1.05 / 0.002  # one request per service time, minus sleep overshoot
