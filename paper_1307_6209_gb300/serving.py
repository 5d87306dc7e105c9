"""Continuous-batching SpMV/SpMMV server over device-resident SELL-C-sigma
matrices (an extension: the paper stops at single products).

Requests (matrix id, block of right-hand sides in pinned host memory) arrive
at any time.  A scheduler thread admits them in arrival order while their
device buffers fit in the HBM budget next to the resident matrices, packs the
admitted ones into one persistent batched launch (sell_batch_create /
sell_batch_run), and keeps up to `streams` batches in flight at once: requests
that arrive while others run on the GPU are admitted as soon as a stream and
memory are free, and their work overlaps on the device.  Each result is
bitwise the same as the request run alone (the per-row arithmetic does not
depend on the batch).  Latency is measured from arrival to the moment the
result is back in host memory (or, for requests whose result stays on the
device, to the completion of the batch on the GPU).
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import sell


@dataclass
class Request:
    rid: int
    mid: int
    X: object                  # pinned host tensor, ncols x k (float64 for F64 matrices, else float32)
    k: int
    t_arrive: float
    t_launch: float = 0.0
    t_done: float = 0.0
    Y: object = None           # result: pinned host tensor, or device tensor (to_host=False)
    done: threading.Event = field(default_factory=threading.Event)
    nbytes: int = 0
    to_host: bool = True

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrive


class Server:
    """Scheduler over resident matrices `mats` (list of SellMatrix)."""

    def __init__(self, mats, hbm_budget_bytes: int, max_batch: int = 128, streams: int = 3,
                 max_wait_s: float = 0.0):
        import torch
        self.torch = torch
        self.mats = list(mats)
        self.resident = sum(h.info.device_bytes for h in self.mats)
        if self.resident > hbm_budget_bytes:
            raise ValueError("resident matrices exceed the HBM budget")
        self.budget = hbm_budget_bytes
        self.max_batch = max_batch
        self.max_wait_s = max_wait_s
        self.inflight_bytes = 0
        self.peak_bytes = self.resident
        self.q = collections.deque()
        self.cv = threading.Condition()
        self.streams = [torch.cuda.Stream() for _ in range(streams)]
        self.free_streams = collections.deque(range(streams))
        self.upload = torch.cuda.Stream()  # kept idle: plan uploads never wait on compute
        self.inflight = []
        self.completed = []
        self.batches = 0
        self.batch_sizes = []
        self._stop = False
        self._rid = 0
        self.thread = None
        self.device = torch.cuda.current_device()

    # ------------------------------------------------------------ client side
    def request_bytes(self, mid: int, k: int) -> int:
        inf = self.mats[mid].info
        es = 8 if inf.store_type == sell.SELL_F64 else 4
        return (inf.ncols + inf.nrows) * k * es

    def submit(self, mid: int, X, to_host: bool = True) -> Request:
        """Queue Y = A_mid X.  X is a pinned host tensor (ncols, or ncols x k);
        the result comes back to pinned host memory, or stays on the device
        (to_host=False) for a consumer that works there."""
        k = 1 if X.dim() == 1 else int(X.shape[1])
        with self.cv:
            r = Request(self._rid, mid, X, k, time.perf_counter(), to_host=to_host)
            r.nbytes = self.request_bytes(mid, k)
            if self.resident + r.nbytes > self.budget:
                raise ValueError("request larger than the HBM budget")
            self._rid += 1
            self.q.append(r)
            self.cv.notify()
        return r

    # ------------------------------------------------------------ scheduler
    def start(self):
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()
        return self

    def stop(self):
        with self.cv:
            self._stop = True
            self.cv.notify()
        if self.thread:
            self.thread.join()

    def _take(self):
        """Admit queued requests in arrival order while they fit."""
        batch = []
        with self.cv:
            while self.q and len(batch) < self.max_batch:
                r = self.q[0]
                if self.resident + self.inflight_bytes + r.nbytes > self.budget:
                    break
                self.q.popleft()
                self.inflight_bytes += r.nbytes
                batch.append(r)
            self.peak_bytes = max(self.peak_bytes, self.resident + self.inflight_bytes)
        return batch

    def _launch(self, batch):
        torch = self.torch
        si = self.free_streams.popleft()
        s = self.streams[si]
        items, bufs = [], []
        now = time.perf_counter()
        with torch.cuda.stream(s):
            for r in batch:
                h = self.mats[r.mid]
                Xd = r.X.to(device=self.device, non_blocking=True)
                shape = (h.info.nrows,) if r.X.dim() == 1 else (h.info.nrows, r.k)
                Yd = torch.empty(shape, dtype=r.X.dtype, device=self.device)
                items.append((h, Xd, Yd, 0))
                bufs.append((r, Xd, Yd))
                r.t_launch = now
        plan = sell.sell_batch_create(items, stream=self.upload)
        plan.run(stream=s)
        with torch.cuda.stream(s):
            for r, Xd, Yd in bufs:
                if r.to_host:
                    r.Y = torch.empty(Yd.shape, dtype=Yd.dtype, pin_memory=True)
                    r.Y.copy_(Yd, non_blocking=True)
                else:
                    r.Y = Yd
            ev = torch.cuda.Event()
            ev.record(s)
        self.inflight.append((si, ev, bufs, plan))
        self.batches += 1
        self.batch_sizes.append(len(batch))

    def _poll(self):
        done_any = False
        for entry in list(self.inflight):
            si, ev, bufs, plan = entry
            if not ev.query():
                continue
            t = time.perf_counter()
            self.inflight.remove(entry)
            plan.free()
            freed = 0
            for r, Xd, Yd in bufs:
                r.t_done = t
                freed += r.nbytes
                r.done.set()
                self.completed.append(r)
            with self.cv:
                self.inflight_bytes -= freed
            self.free_streams.append(si)
            done_any = True
        return done_any

    def _loop(self):
        self.torch.cuda.set_device(self.device)
        while True:
            self._poll()
            launched = False
            if self.free_streams:
                if self.max_wait_s and self.inflight:
                    # optional small wait to gather more requests into one launch
                    with self.cv:
                        if len(self.q) < self.max_batch:
                            self.cv.wait(timeout=self.max_wait_s)
                batch = self._take()
                if batch:
                    self._launch(batch)
                    launched = True
            with self.cv:
                if self._stop and not self.q and not self.inflight:
                    return
                if not launched and not self.inflight and not self.q:
                    self.cv.wait(timeout=0.01)
            if not launched and self.inflight:
                time.sleep(2e-5)

    # ------------------------------------------------------------ reporting
    def stats(self):
        lat = np.array([r.latency for r in self.completed]) if self.completed else np.zeros(1)
        return {"requests": len(self.completed), "batches": self.batches,
                "mean_batch": float(np.mean(self.batch_sizes)) if self.batch_sizes else 0.0,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3), "peak_hbm_bytes": int(self.peak_bytes),
                "budget_bytes": int(self.budget)}


def poisson_load(server: Server, rate_hz: float, duration_s: float, make_request, seed: int = 0,
                 to_host: bool = True):
    """Submit requests with exponential inter-arrival times for duration_s;
    make_request(rng) -> (mid, pinned X).  Returns the submitted requests."""
    rng = np.random.default_rng(seed)
    reqs = []
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
        reqs.append(server.submit(mid, X, to_host=to_host))
    return reqs
