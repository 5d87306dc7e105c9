"""Python face of the native continuous-batching server (sell_server_* in
include/sell.h; the scheduler, admission, batching and stream handling run in
the C++ library).

Requests (matrix id, block of right-hand sides in pinned host memory) are
queued from any thread.  The library's scheduler thread admits them in arrival
order while their device footprint (x block, y block, long-row scratch) fits
in an arena of budget - resident bytes, packs the admitted ones into one
batched launch on a free stream and keeps up to `streams` batches in flight,
so requests that arrive while others run are admitted as soon as a stream and
memory are free and their work overlaps on the device.  Each result is
bitwise the same as the request run alone.  Latency is measured by the
library from arrival to the moment the request's batch has completed on the
GPU (results copied back into the request's pinned host buffer, or left on
the device).
"""
from __future__ import annotations

import gc
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import sell


class _DeviceArray:
    """__cuda_array_interface__ view of a device result (no copy)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


@dataclass
class Request:
    server: "Server"
    rid: int
    mid: int
    X: object                  # pinned host tensor, ncols (k = 1) or ncols x k
    k: int
    to_host: bool
    Y: object = None           # pinned host result (to_host), else set by result()
    t_arrive: float = 0.0
    t_launch: float = 0.0
    t_done: float = 0.0
    batch: int = 0
    finished: bool = False
    released: bool = False
    _lock: threading.Lock = field(default_factory=threading.Lock)

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrive

    def wait(self, timeout: float = 60.0) -> "Request":
        """Block until the request has completed (raises on timeout or error)."""
        with self._lock:
            if not self.finished:
                info = sell.sell_server_wait(self.server.handle, self.rid, timeout)
                self.t_arrive, self.t_launch, self.t_done = info.t_arrive, info.t_launch, info.t_done
                self.batch = info.batch
                self.finished = True
                self.server._record(self)
        return self

    def result(self):
        """The device result (to_host=False) as a torch tensor view, valid until release()."""
        import torch
        self.wait()
        if self.to_host:
            return self.Y
        ptr = sell.sell_server_result(self.server.handle, self.rid)
        inf = self.server.mats[self.mid].info
        shape = (inf.nrows,) if self.X.dim() == 1 else (inf.nrows, self.k)
        typestr = "<f8" if inf.store_type == sell.SELL_F64 else "<f4"
        return torch.as_tensor(_DeviceArray(ptr, shape, typestr), device="cuda")

    def release(self):
        """Return a device result's memory to the server."""
        if not self.to_host and not self.released:
            self.wait()
            sell.sell_server_release(self.server.handle, self.rid)
            self.released = True


class Server:
    """Native server over resident matrices `mats` (list of SellMatrix)."""

    def __init__(self, mats, hbm_budget_bytes: int, max_batch: int = 128, streams: int = 6, size_ratio: int = 0,
                 max_batch_work: int = 0):
        self.mats = list(mats)
        self.resident = sum(h.info.device_bytes for h in self.mats)
        if self.resident >= hbm_budget_bytes:
            raise ValueError("resident matrices fill the HBM budget")
        self.budget = int(hbm_budget_bytes)
        self.handle = sell.sell_server_create(self.mats, self.budget, max_batch, streams, size_ratio, max_batch_work)
        self._done = []
        self._done_lock = threading.Lock()
        self._pending = {}  # id -> Request, until collected

    # -------------------------------------------------------------- client
    def request_bytes(self, mid: int, k: int) -> int:
        """The x and y blocks of a request (the library adds long-row scratch)."""
        inf = self.mats[mid].info
        es = 8 if inf.store_type == sell.SELL_F64 else 4
        return (inf.ncols + inf.nrows) * k * es

    def submit(self, mid: int, X, to_host: bool = True) -> Request:
        """Queue Y = A_mid X.  X is a pinned host tensor (ncols, or ncols x k);
        the result comes back to a pinned host tensor (to_host), or stays on
        the device until Request.release()."""
        import torch
        k = 1 if X.dim() == 1 else int(X.shape[1])
        Y = None
        if to_host:
            inf = self.mats[mid].info
            shape = (inf.nrows,) if X.dim() == 1 else (inf.nrows, k)
            Y = torch.empty(shape, dtype=X.dtype, pin_memory=True)
        # registered under the lock that next() takes to look a request up, so
        # a request that completes at once is never delivered unknown
        with self._done_lock:
            try:
                rid = sell.sell_server_submit(self.handle, mid, X.data_ptr(), k,
                                              Y.data_ptr() if Y is not None else None)
            except sell.SellError as e:
                raise ValueError(str(e)) from e
            r = Request(self, rid, mid, X, k, to_host, Y=Y)
            self._pending[rid] = r
        return r

    def next(self, timeout: float = 60.0) -> Request:
        """The next completed request, in completion order (raises SellError
        with SELL_ETIMEOUT when none completes in time)."""
        rid, info = sell.sell_server_next(self.handle, timeout)
        with self._done_lock:
            r = self._pending.get(rid)
        with r._lock:
            r.t_arrive, r.t_launch, r.t_done = info.t_arrive, info.t_launch, info.t_done
            r.batch = info.batch
            r.finished = True
        self._record(r)
        return r

    def work(self, mid: int, k: int) -> int:
        """A request's work as the server measures it: stored elements x k."""
        return int(self.mats[mid].info.stored) * int(k)

    def _record(self, r: Request):
        with self._done_lock:
            self._done.append((r.t_arrive, r.t_launch, r.t_done, r.batch, self.work(r.mid, r.k)))
            self._pending.pop(r.rid, None)

    # ----------------------------------------------------------- lifecycle
    def start(self):
        return self  # the scheduler thread runs from creation on

    def stop(self):
        if self.handle:
            sell.sell_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass

    # ----------------------------------------------------------- reporting
    def stats(self, split_work: int = 0):
        """Counters and latency percentiles; with a work threshold (stored
        elements x k), also per size class: "small" (work <= threshold) and
        "large"."""
        st = sell.sell_server_stats(self.handle) if self.handle else {}
        with self._done_lock:
            d = np.array(self._done, dtype=np.float64) if self._done else np.zeros((1, 5))
        lat = d[:, 2] - d[:, 0]
        out = {"requests": int(st.get("requests", len(self._done))), "batches": int(st.get("batches", 0)),
               "mean_batch": float(st["batched_requests"] / max(1, st["batches"])) if st else 0.0,
               "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
               "mean_ms": float(lat.mean() * 1e3), "peak_hbm_bytes": int(st.get("peak_bytes", 0)),
               "budget_bytes": self.budget}
        split = int(split_work)
        if split > 0 and self._done:
            for name, sel in (("small", d[:, 4] <= split), ("large", d[:, 4] > split)):
                if sel.any():
                    out[name] = {"requests": int(sel.sum()), "p50_ms": float(np.percentile(lat[sel], 50) * 1e3),
                                 "p99_ms": float(np.percentile(lat[sel], 99) * 1e3)}
        return out


class _Consumer:
    """A client thread that takes requests as they complete (completion
    order, sell_server_next) and releases device results at once."""

    def __init__(self, server: Server):
        self.server = server
        self.submitted = 0
        self.collected = 0
        self.closed = False
        self.errors = []
        self.th = threading.Thread(target=self._run, daemon=True)
        self.th.start()

    def _run(self):
        last = time.perf_counter()
        while not (self.closed and self.collected >= self.submitted):
            try:
                r = self.server.next(0.05)
                last = time.perf_counter()
            except sell.SellError as e:
                if e.status == sell.SELL_ETIMEOUT:
                    if self.collected < self.submitted and time.perf_counter() - last > 120.0:
                        self.errors.append(TimeoutError("no request completed for 120 s"))
                        return
                    continue
                self.errors.append(e)
                return
            except Exception as e:  # surfaced by finish()
                self.errors.append(e)
                return
            try:
                r.release()
            except Exception as e:
                self.errors.append(e)
            self.collected += 1

    def put(self, r):
        self.submitted += 1

    def finish(self):
        self.closed = True
        self.th.join()
        if self.errors:
            raise self.errors[0]


class _NoGC:
    """Python's cyclic garbage collector paused for a load run (a collection
    pass over a large heap stalls the submitting thread for milliseconds and
    turns Poisson arrivals into bursts)."""

    def __enter__(self):
        gc.collect()
        self.was = gc.isenabled()
        gc.disable()

    def __exit__(self, *exc):
        if self.was:
            gc.enable()


def burst_load(server: Server, n: int, make_request, seed: int = 0, to_host: bool = True):
    """Submit n requests at once; returns (requests, seconds until the last
    completed)."""
    with _NoGC():
        return _burst_load(server, n, make_request, seed, to_host)


def _burst_load(server, n, make_request, seed, to_host):
    rng = np.random.default_rng(seed)
    c = _Consumer(server)
    t0 = time.perf_counter()
    reqs = []
    for _ in range(n):
        r = server.submit(*make_request(rng), to_host=to_host)
        reqs.append(r)
        c.put(r)
    c.finish()
    return reqs, time.perf_counter() - t0


def poisson_load(server: Server, rate_hz: float, duration_s: float, make_request, seed: int = 0,
                 to_host: bool = True):
    """Submit requests with exponential inter-arrival times for duration_s;
    make_request(rng) -> (mid, pinned X); a consumer thread takes the
    results as they arrive.  Returns the requests, all complete."""
    with _NoGC():
        return _poisson_load(server, rate_hz, duration_s, make_request, seed, to_host)


def _poisson_load(server, rate_hz, duration_s, make_request, seed, to_host):
    rng = np.random.default_rng(seed)
    reqs = []
    c = _Consumer(server)
    t0 = time.perf_counter()
    t_next = t0
    while True:
        t_next += rng.exponential(1.0 / rate_hz)
        if t_next - t0 > duration_s:
            break
        while True:
            now = time.perf_counter()
            if now >= t_next:
                break
            time.sleep(min(t_next - now, 1e-4))
        mid, X = make_request(rng)
        r = server.submit(mid, X, to_host=to_host)
        reqs.append(r)
        c.put(r)
    c.finish()
    return reqs


def closed_loop(server: Server, outstanding: int, duration_s: float, make_request, seed: int = 0,
                to_host: bool = True):
    """Saturated throughput in steady state: keep `outstanding` requests
    queued or running for duration_s (each completion submits the next
    request), then drain.  Returns (requests completed within the window,
    window seconds); the caller divides."""
    with _NoGC():
        return _closed_loop(server, outstanding, duration_s, make_request, seed, to_host)


def _closed_loop(server, outstanding, duration_s, make_request, seed, to_host):
    rng = np.random.default_rng(seed)
    live = 0
    for _ in range(outstanding):
        server.submit(*make_request(rng), to_host=to_host)
        live += 1
    t0 = time.perf_counter()
    done = 0
    while True:
        r = server.next(60.0)
        r.release()
        live -= 1
        if time.perf_counter() - t0 >= duration_s:
            break
        done += 1
        server.submit(*make_request(rng), to_host=to_host)
        live += 1
    t1 = time.perf_counter()
    while live > 0:
        server.next(60.0).release()
        live -= 1
    return done, t1 - t0
