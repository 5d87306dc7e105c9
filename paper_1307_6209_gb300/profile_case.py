"""Run one configured SpMV / SpMMV case, for profilers and quick timing.

    python -m paper_1307_6209_gb300.profile_case --matrix stencil27 --n 120 --store bf16 \\
        --C 32 --sigma 1 --block 128 --unroll 8 --pipeline 1 --k 1 --reps 5

builds the synthetic matrix on the device, converts it with the given (C,
sigma) and storage type, fixes the launch, runs `--warmup` untimed and
`--reps` timed products on one stream (CUDA events) and prints one JSON line
with the kernel's average time, GF/s and algorithmic GB/s.  Everything runs
through the C ABI; nothing is tuned.

    python -m paper_1307_6209_gb300.profile_case --batch 64 --store f32 --C 32 --sigma 4096 --k 1

runs a batch plan instead (sell_batch_create / sell_batch_run): `--batch`
matrices with rows uniform in [1000, 200000] (seeded), even ones banded
(bandwidth 64, 7-30 entries per row) and odd ones lognormal (`--kinds banded`
or `lognormal`: one kind only), all in the given (C, sigma) and storage type,
each with its own k right-hand sides.

    python -m paper_1307_6209_gb300.profile_case --measure gathers   (or copies)

measures the random-gather rates of the load/store path and of TMA gather4,
or how host-to-device copies on two streams share the copy engine.
"""
from __future__ import annotations

import argparse
import json


def main(argv=None):
    import torch

    from . import model, sell, synth

    p = argparse.ArgumentParser()
    p.add_argument("--matrix", choices=["stencil27", "lognormal", "dense", "long_row", "banded"], default="stencil27")
    p.add_argument("--n", type=int, default=120, help="grid edge (stencil27) or rows")
    p.add_argument("--store", choices=["f64", "f32", "bf16"], default="f64")
    p.add_argument("--C", type=int, default=32)
    p.add_argument("--sigma", type=int, default=1)
    p.add_argument("--block", type=int, default=128)
    p.add_argument("--unroll", type=int, default=4)
    p.add_argument("--pipeline", type=int, default=0)
    p.add_argument("--k", type=int, default=1)
    p.add_argument("--compensated", action="store_true")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--reps", type=int, default=5)
    p.add_argument("--batch", type=int, default=0, help="run a batch plan of this many matrices")
    p.add_argument("--kinds", choices=["mixed", "banded", "lognormal"], default="mixed",
                   help="batch matrices: alternating banded / lognormal, or one kind only")
    p.add_argument("--tile", type=int, default=0, help="batch block size (64, 128, 256; 0 keeps the default)")
    p.add_argument("--measure", choices=["gathers", "copies"], default=None,
                   help="gathers: random-gather rates of the load/store path and of TMA gather4 "
                        "(sell_bench_gather / sell_bench_gather4); copies: a small host-to-device copy "
                        "issued after a large one on another stream")
    a = p.parse_args(argv)
    if a.measure == "gathers":
        return run_gathers()
    if a.measure == "copies":
        return run_copies()
    if a.batch > 0:
        return run_batch(a)

    if a.matrix == "stencil27":
        A = synth.stencil27_device(a.n, perturb=0.1, seed=0)
    elif a.matrix == "lognormal":
        A = synth.lognormal_device(a.n, seed=0)
    elif a.matrix == "dense":
        A = synth.dense_device(a.n)
    elif a.matrix == "long_row":
        A = synth.long_row_device(a.n, a.n, short_len=3, at=a.n // 3)
    else:
        A = synth.banded_device(a.n, seed=0)
    st = {"f64": sell.SELL_F64, "f32": sell.SELL_F32, "bf16": sell.SELL_BF16}[a.store]
    dt = torch.float64 if st == sell.SELL_F64 else torch.float32
    s = torch.cuda.Stream()
    h = sell.sell_build(A, C=a.C, sigma=a.sigma, store_type=st, stream=s)
    sell.sell_set_launch(h, a.block, a.unroll, a.pipeline)
    g = torch.Generator("cuda").manual_seed(0)
    X = torch.rand((A.ncols, a.k), dtype=dt, device="cuda", generator=g) * 2 - 1
    Y = torch.empty((A.nrows, a.k), dtype=dt, device="cuda")
    x1, y1 = X[:, 0].contiguous(), Y[:, 0].contiguous()
    flags = sell.SELL_SPMV_COMPENSATED if a.compensated else 0

    def step():
        if a.k == 1:
            sell.sell_spmv(h, x1, y1, flags=flags, stream=s)
        else:
            sell.sell_spmmv(h, X, Y, flags=flags, stream=s)

    for _ in range(a.warmup):
        step()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.reps)]
    for e0, e1 in ev:
        e0.record(s)
        step()
        e1.record(s)
    torch.cuda.synchronize()
    sell.sell_check(h, stream=s)
    us = sum(e0.elapsed_time(e1) for e0, e1 in ev) * 1e3 / a.reps
    inf = h.info
    vb = {sell.SELL_F64: 8, sell.SELL_F32: 4}.get(st, 2)
    xb = 8 if st == sell.SELL_F64 else 4
    alg = model.algorithmic_bytes(inf.nrows, inf.ncols, inf.nnz, inf.nchunks, a.C, vb, xb, inf.has_perm, k=a.k)
    print(json.dumps({"matrix": a.matrix, "n": a.n, "nrows": inf.nrows, "nnz": inf.nnz, "store": a.store,
                      "C": a.C, "sigma": a.sigma, "beta": round(inf.beta, 6), "block": a.block,
                      "unroll": a.unroll, "pipeline": a.pipeline, "k": a.k, "us": round(us, 3),
                      "gflops": round(2.0 * inf.nnz * a.k / us / 1e3, 1),
                      "algorithmic_gbs": round(alg / us / 1e3, 1), "value_bytes": vb}))
    h.free()
    return 0


def run_batch(a):
    import numpy as np
    import torch

    from . import model, sell, synth

    st = {"f64": sell.SELL_F64, "f32": sell.SELL_F32, "bf16": sell.SELL_BF16}[a.store]
    dt = torch.float64 if st == sell.SELL_F64 else torch.float32
    vb = {sell.SELL_F64: 8, sell.SELL_F32: 4}.get(st, 2)
    xb = 8 if st == sell.SELL_F64 else 4
    s = torch.cuda.Stream()
    sizes = np.random.default_rng(0).integers(1000, 200001, a.batch)
    g = torch.Generator("cuda").manual_seed(0)
    items, alg, nnz, stored = [], 0, 0, 0
    for i, n in enumerate(sizes):
        banded = a.kinds == "banded" or (a.kinds == "mixed" and i % 2 == 0)
        gen = synth.banded_device if banded else synth.lognormal_device
        A = gen(int(n), seed=i)
        h = sell.sell_build(A, C=a.C, sigma=a.sigma, store_type=st, stream=s)
        inf = h.info
        shp_x = (inf.ncols,) if a.k == 1 else (inf.ncols, a.k)
        shp_y = (inf.nrows,) if a.k == 1 else (inf.nrows, a.k)
        items.append((h, torch.rand(shp_x, dtype=dt, device="cuda", generator=g) * 2 - 1,
                      torch.empty(shp_y, dtype=dt, device="cuda"), 0))
        alg += model.algorithmic_bytes(inf.nrows, inf.ncols, inf.nnz, inf.nchunks, a.C, vb, xb, inf.has_perm, k=a.k)
        nnz += inf.nnz
        stored += inf.stored
        del A
    plan = sell.sell_batch_create(items, stream=s)
    if a.tile:
        plan.set_launch(a.tile)
    for _ in range(a.warmup):
        plan.run(stream=s)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.reps)]
    for e0, e1 in ev:
        e0.record(s)
        plan.run(stream=s)
        e1.record(s)
    torch.cuda.synchronize()
    us = sum(e0.elapsed_time(e1) for e0, e1 in ev) * 1e3 / a.reps
    print(json.dumps({"batch": a.batch, "kinds": a.kinds, "tile": a.tile, "rows": int(sizes.sum()), "nnz": nnz,
                      "stored": stored,
                      "beta": round(nnz / max(stored, 1), 6), "store": a.store, "C": a.C, "sigma": a.sigma,
                      "k": a.k, "us": round(us, 3), "gflops": round(2.0 * nnz * a.k / us / 1e3, 1),
                      "algorithmic_bytes": alg, "algorithmic_gbs": round(alg / us / 1e3, 1),
                      "value_bytes": vb}))
    plan.free()
    for h, _, _, _ in items:
        h.free()
    return 0


def _best_ms(fn, stream, reps=5):
    import torch
    fn()
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def run_gathers():
    """Random sectors per second from an L2-resident x through the load/store
    path (8-byte words) and through TMA gather4 (16-byte rows, four per copy)."""
    import torch

    from . import sell
    sell.load()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    s = torch.cuda.Stream()
    out = []
    for nw in (2_000_000, 8_000_000):
        x = torch.ones(nw, dtype=torch.int64, device="cuda")
        grid, iters = sms * 8, 64
        sink = torch.zeros(grid * 256, dtype=torch.float64, device="cuda")
        ms = _best_ms(lambda: sell.sell_bench_gather(x, nw, sink, grid, iters, stream=s), s)
        out.append({"kernel": "k_gather", "n_words": nw, "grid": grid, "threads": 256, "iters": iters,
                    "G_per_s": round(grid * 256 * iters * 8 / ms / 1e6, 1)})
        for bps in (2, 4, 7):
            for iters in (64, 256):
                grid = sms * bps
                sink = torch.zeros(grid * 128 + 1, dtype=torch.float64, device="cuda")
                ms = _best_ms(lambda: sell.sell_bench_gather4(x, nw, sink, grid, iters, stream=s), s)
                out.append({"kernel": "k_gather4", "n_words": nw, "grid": grid, "threads": 128, "iters": iters,
                            "G_per_s": round(grid * 128 * iters * 4 / ms / 1e6, 1),
                            "wait_gave_up": bool(sink[-1].item() != 0)})
        del x
    print(json.dumps(out))
    return 0


def run_copies():
    """A 64 KB host-to-device copy issued right after a 256 MB one on another
    stream: when does it complete?  (And the small copy alone, and two large
    copies on two streams.)"""
    import torch
    big_h = torch.rand(32 * 2 ** 20, dtype=torch.float64).pin_memory()
    big_d = torch.empty_like(big_h, device="cuda")
    small_h = torch.rand(8192, dtype=torch.float64).pin_memory()
    small_d = torch.empty_like(small_h, device="cuda")
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    out = {"trials": []}
    for _ in range(3):
        torch.cuda.synchronize()
        e0, ea, eb = ev(), ev(), ev()
        e0.record(sa)
        with torch.cuda.stream(sa):
            big_d.copy_(big_h, non_blocking=True)
        ea.record(sa)
        sb.wait_event(e0)
        with torch.cuda.stream(sb):
            small_d.copy_(small_h, non_blocking=True)
        eb.record(sb)
        torch.cuda.synchronize()
        out["trials"].append({"large_done_ms": round(e0.elapsed_time(ea), 3),
                              "small_done_ms": round(e0.elapsed_time(eb), 3)})
    e0, e1 = ev(), ev()
    e0.record(sb)
    with torch.cuda.stream(sb):
        small_d.copy_(small_h, non_blocking=True)
    e1.record(sb)
    torch.cuda.synchronize()
    out["small_alone_ms"] = round(e0.elapsed_time(e1), 4)
    big_h2 = torch.rand(32 * 2 ** 20, dtype=torch.float64).pin_memory()
    big_d2 = torch.empty_like(big_h2, device="cuda")
    e0, e1, e2 = ev(), ev(), ev()
    e0.record(sa)
    sb.wait_event(e0)
    with torch.cuda.stream(sa):
        big_d.copy_(big_h, non_blocking=True)
    with torch.cuda.stream(sb):
        big_d2.copy_(big_h2, non_blocking=True)
    e1.record(sa)
    e2.record(sb)
    torch.cuda.synchronize()
    out["two_large_done_ms"] = [round(e0.elapsed_time(e1), 3), round(e0.elapsed_time(e2), 3)]
    # a host-to-device and a device-to-host copy of 256 MB at once, on two streams
    back_h = torch.empty_like(big_h).pin_memory()
    torch.cuda.synchronize()
    e0, e1, e2 = ev(), ev(), ev()
    e0.record(sa)
    sb.wait_event(e0)
    with torch.cuda.stream(sa):
        big_d.copy_(big_h, non_blocking=True)
    with torch.cuda.stream(sb):
        back_h.copy_(big_d2, non_blocking=True)
    e1.record(sa)
    e2.record(sb)
    torch.cuda.synchronize()
    out["h2d_and_d2h_done_ms"] = [round(e0.elapsed_time(e1), 3), round(e0.elapsed_time(e2), 3)]
    out["large_gbs"] = round(big_h.numel() * 8 / (out["trials"][-1]["large_done_ms"] * 1e-3) / 1e9, 1)
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
