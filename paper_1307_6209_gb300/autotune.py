"""Autotuner for SELL-C-sigma on GB300: picks C, sigma, the block size, the
unroll depth and the software pipelining of the SpMV by measurement.

The paper leaves the choice of sigma and of the threads per row to future
work (Sec. 6) and notes that the best sigma is matrix dependent (Sec. 3.4,
Sec. 5.3).  Stage 1 builds every (C, sigma) candidate and times the SpMV with
the default launch; stage 2 sweeps (block, unroll, pipeline) on the best
formats (software pipelining at every number of right-hand sides, bulk
staging for single right-hand sides, where they exist).  All
timing goes through the C ABI (CUDA events on the given stream).  Results are
cached in a JSON file keyed by a matrix signature (sizes, longest row, the
coefficient of variation of Eq. "cv", storage type, right-hand sides).
"""
from __future__ import annotations

import json
import os
import time
from dataclasses import asdict, dataclass, field

from . import sell

DEFAULT_CACHE = os.environ.get("SELL_AUTOTUNE_CACHE",
                               os.path.join(os.path.expanduser("~"), ".cache", "sellcs", "autotune.json"))


@dataclass
class Choice:
    C: int
    sigma: int
    block: int
    unroll: int
    us: float
    gflops: float
    pipeline: int = 0


@dataclass
class TuneResult:
    best: Choice
    formats: list = field(default_factory=list)  # stage 1: (C, sigma, beta, us, build_ms)
    launches: list = field(default_factory=list)  # stage 2: (C, sigma, block, unroll, pipeline, us)
    cached: bool = False


def _time(fn, stream, reps):
    import torch
    for _ in range(3):
        fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) * 1e3 / reps  # microseconds


def signature(info: "sell.Info", store_type: int, k: int) -> str:
    return (f"n{info.nrows}_m{info.ncols}_nnz{info.nnz}_max{info.max_row_len}_z{info.zeta:.3f}"
            f"_t{store_type}_k{k}")


def _load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def _save_cache(path, data):
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1)
        os.replace(tmp, path)
    except OSError:
        pass


def tune(A, store_type: int = sell.SELL_F64, k: int = 1, Cs=(32, 64, 128), sigmas=None,
         blocks=(128, 256, 512), unrolls=(1, 2, 4, 8), pipelines=(0, 1, 2), keep: int = 2, reps: int = 30,
         stream=None,
         cache: str | None = DEFAULT_CACHE, use_cache: bool = True) -> TuneResult:
    """Tune the SpMV (k = 1) or SpMMV (k > 1) of CSR matrix A (host numpy or
    device torch arrays).  Returns the best (C, sigma, block, unroll, pipeline)."""
    import torch

    stream = stream or torch.cuda.current_stream()
    nrows = int(A.nrows)
    # sigma = N may coincide with a fixed point of the sweep (N = 256, 4096)
    sigmas = tuple(dict.fromkeys(sigmas or (1, 256, 4096, max(nrows, 1))))
    dt = torch.float64 if store_type == sell.SELL_F64 else torch.float32
    X = torch.rand((int(A.ncols), k), dtype=dt, device="cuda") * 2 - 1
    Y = torch.empty((nrows, k), dtype=dt, device="cuda")
    x1, y1 = X[:, 0].contiguous(), Y[:, 0].contiguous()
    flops = 2.0 * float(A.rpt[-1]) * k

    def product(h):
        if k == 1:
            sell.sell_spmv(h, x1, y1, stream=stream)
        else:
            sell.sell_spmmv(h, X, Y, stream=stream)

    key = None
    formats = []
    built = {}
    for C in Cs:
        for s in sigmas:
            t0 = time.perf_counter()
            h = sell.sell_build(A, C=C, sigma=s, store_type=store_type, stream=stream)
            bms = (time.perf_counter() - t0) * 1e3
            if key is None:
                key = signature(h.info, store_type, k)
                if use_cache and cache:
                    hit = _load_cache(cache).get(key)
                    if hit:
                        h.free()
                        return TuneResult(best=Choice(**hit), cached=True)
            us = _time(lambda: product(h), stream, reps)
            formats.append({"C": C, "sigma": s, "beta": h.info.beta, "us": us, "build_ms": bms})
            built[(C, s)] = h
    formats.sort(key=lambda r: r["us"])
    launches = []
    best = None
    for r in formats[:keep]:
        h = built[(r["C"], r["sigma"])]
        for b in blocks:
            for u in unrolls:
                for p in pipelines:
                    if (p == 1 and k > 2) or (p == 2 and k > 1):
                        continue  # modes 1 and 2 exist for k <= 2 and k = 1
                    try:
                        sell.sell_set_launch(h, b, u, p)
                    except sell.SellError:
                        continue  # e.g. mode 2 with a C it does not take
                    us = _time(lambda: product(h), stream, reps)
                    launches.append({"C": r["C"], "sigma": r["sigma"], "block": b, "unroll": u, "pipeline": p,
                                     "us": us})
                    if best is None or us < best.us:
                        best = Choice(r["C"], r["sigma"], b, u, us, flops / us / 1e3, p)
    for h in built.values():
        h.free()
    if cache:
        data = _load_cache(cache)
        data[key] = asdict(best)
        _save_cache(cache, data)
    return TuneResult(best=best, formats=formats, launches=launches)


def build_tuned(A, choice: Choice, store_type: int = sell.SELL_F64, stream=None) -> "sell.SellMatrix":
    """Build the handle the tuner chose and apply its launch shape."""
    h = sell.sell_build(A, C=choice.C, sigma=choice.sigma, store_type=store_type, stream=stream)
    sell.sell_set_launch(h, choice.block, choice.unroll, choice.pipeline)
    return h


def tune_batch(samples, store_type: int = sell.SELL_F32, Cs=(32, 64), sigmas=(1, 32, 256, 2048, 4096, 1 << 30),
               reps: int = 10, stream=None):
    """Pick (C, sigma) for a class of matrices by the throughput of a batch.

    Each candidate builds every sample matrix and times one batched launch
    (sell_batch_create / sell_batch_run) over all of them.  A single small
    matrix is latency-bound and would favour formats that move more bytes;
    in a batch, the bytes count: with unsorted chunks the row-length skip
    saves instructions but not DRAM sectors, so the padding of Eq. "beta" is
    read anyway.  Returns (best {"C", "sigma", "us"}, list of all candidates).
    """
    import torch

    stream = stream or torch.cuda.current_stream()
    dt = torch.float64 if store_type == sell.SELL_F64 else torch.float32
    best, table = None, []
    for C in Cs:
        for sg in sigmas:
            hs = [sell.sell_build(A, C=C, sigma=sg, store_type=store_type, stream=stream) for A in samples]
            items = [(h, torch.rand(h.info.ncols, dtype=dt, device="cuda"),
                      torch.empty(h.info.nrows, dtype=dt, device="cuda"), 0) for h in hs]
            plan = sell.sell_batch_create(items, stream=stream)
            us = _time(lambda: plan.run(stream=stream), stream, reps)
            table.append({"C": C, "sigma": sg, "us": us})
            if best is None or us < best["us"]:
                best = {"C": C, "sigma": sg, "us": us}
            plan.free()
            for h in hs:
                h.free()
    return best, table


def tune_plan(items, k: int, tiles=(64, 128, 256), rhs=(8, 4), reps: int = 10, stream=None):
    """Pick the launch of a whole batch plan by timing it: the block size
    (rows per work unit, sell_batch_set_launch) and, for k >= 4 right-hand
    sides, the widest block of right-hand sides (SELL_SPMV_RHS_BLOCK*).
    Neither changes any result.  items: (handle, X, Y, flags) as for
    sell_batch_create.  Returns (best {"tile", "rhs", "us"}, all candidates)."""
    import torch

    stream = stream or torch.cuda.current_stream()
    flag = {8: 0, 4: sell.SELL_SPMV_RHS_BLOCK4, 2: sell.SELL_SPMV_RHS_BLOCK2, 1: sell.SELL_SPMV_RHS_BLOCK1}
    best, table = None, []
    for w in (rhs if k >= 4 else (8,)):
        plan = sell.sell_batch_create([(h, X, Y, fl | flag[w]) for h, X, Y, fl in items], stream=stream)
        for t in tiles:
            plan.set_launch(t)
            us = _time(lambda: plan.run(stream=stream), stream, reps)
            table.append({"tile": t, "rhs": w, "us": us})
            if best is None or us < best["us"]:
                best = {"tile": t, "rhs": w, "us": us}
        plan.free()
    return best, table
