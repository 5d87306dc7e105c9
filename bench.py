#!/usr/bin/env python
"""SELL-C-sigma SpMV benchmark (GB300, sm_103a).

Headline workload: the 27-point stencil on a 200^3 grid (N = 8,000,000 rows,
213,847,192 nonzeros), binary64 values 26 / -1 times 1 + 0.1 U(-1, 1), generated
on the device; x ~ U[-1, 1] (seed 0).  It is the largest configuration that
fits one GPU.  The autotuner picks C, sigma and the launch shape; a step is
one binary64 SpMV y = A x with the tuned choice.

The line also reports, for the same matrix, binary32 and bfloat16 storage
("FP64 vs mixed"), SpMMV and the end-to-end rate through host buffers; the
co-bounds (HBM read bandwidth, L2 random-gather rate, FP64 FMA rate); the
lognormal N = 2,000,000 matrix with its C x sigma sweep; the 5-point
Laplacian; the pathological shapes of Sec. 5.2; the 512-matrix batch; the
64-matrix serving run; and it ends with a compact summary of every figure.

One JSON line is printed by rank 0.  Under torchrun every rank runs its own
replica of the workload on its own GPU (independent problems, no data-path
collective: weak scaling); the step time is the maximum over ranks.

--impl reference runs the CPU oracle (CRS SpMV in binary64, OpenMP on the
host cores) on a bounded row sample of the same workload per step instead.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L2_BYTES = 129 * 2 ** 20
FALLBACK_HBM_GBS = 6800.0
# the same metric string on both arms (the reference arm times the CPU oracle)
METRIC = "SpMV GF/s (FP64)"

KERNEL_SOURCES = ["paper_1307_6209_gb300/csrc/sell_spmv_impl.cuh", "paper_1307_6209_gb300/csrc/sell_spmv_f64.cu",
                  "paper_1307_6209_gb300/csrc/sell_device.cuh", "paper_1307_6209_gb300/csrc/sell_rowdot.cuh",
                  "paper_1307_6209_gb300/csrc/sell_spmv_bulk.cuh"]


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["stencil27", "lognormal", "laplace"], default="stencil27")
    p.add_argument("--n", type=int, default=None, help="grid edge (stencils) or rows (lognormal)")
    p.add_argument("--C", type=int, default=None)
    p.add_argument("--sigma", type=int, default=None)
    p.add_argument("--block", type=int, default=None, help="fix the launch block instead of tuning it")
    p.add_argument("--unroll", type=int, default=None, help="fix the unroll instead of tuning it")
    p.add_argument("--pipeline", type=int, default=None, help="fix the launch mode (0, 1, 2) instead of tuning it")
    p.add_argument("--no-sweep", action="store_true")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--no-extras", action="store_true", help="skip every section but the headline")
    p.add_argument("--section", choices=["serving"], default=None,
                   help="run one extra section alone and print its JSON object (the serving section runs so, in a "
                        "process of its own)")
    p.add_argument("--shard", choices=["replicas", "rows"], default="replicas",
                   help="replicas: every rank multiplies its own copy (weak scaling); rows: the ranks split one "
                        "matrix by rows, one allgather of x per step (strong scaling)")
    return p.parse_args()


# ------------------------------------------------------------------ workloads
def workload(args):
    """The workload's description, tuning grid and generators: `device()`
    returns the CSR on the GPU (torch arrays), `host(rows)` the CSR (or its
    first `rows` rows) in numpy."""
    from paper_1307_6209_gb300 import synth
    if args.workload == "stencil27":
        n = args.n or 200
        N, nnz = n ** 3, (3 * n - 2) ** 3
        return {"name": "stencil27", "nrows": N, "nnz": nnz,
                "desc": f"27-point stencil on a {n}^3 grid (N={N}, nnz={nnz}), FP64 values 26/-1 times "
                        f"1+0.1*U(-1,1), x ~ U[-1,1] seed 0",
                "grid": [(32, 1), (32, 4096), (64, 1), (128, 1)],
                "device": lambda: synth.stencil27_device(n, perturb=0.1, seed=0),
                "host": lambda rows=None: synth.stencil27(n, perturb=0.1, seed=0, rows=rows)}
    if args.workload == "lognormal":
        n = args.n or 2_000_000
        return {"name": "lognormal", "nrows": n, "nnz": None,
                "desc": f"lognormal random N={n} (row length mean 16, log-sd 1.2, cap 2000), FP64",
                "grid": [(C, s) for C in (32, 64, 128) for s in (1, 256, 4096, n)],
                "device": None,
                "host": lambda rows=None: synth.lognormal(n, mean=16.0, sigma_ln=1.2, cap=2000, seed=0)}
    n = args.n or 64
    return {"name": "laplace", "nrows": n * n, "nnz": None,
            "desc": f"5-point Laplacian on a {n}x{n} grid, FP64", "grid": [(32, 1)], "device": None,
            "host": lambda rows=None: synth.laplace2d(n)}


def to_device(A):
    import torch
    return type(A)(A.nrows, A.ncols, torch.from_numpy(A.rpt).cuda(), torch.from_numpy(A.col).cuda(),
                   torch.from_numpy(A.val).cuda())


def to_host(A):
    return type(A)(A.nrows, A.ncols, A.rpt.cpu().numpy(), A.col.cpu().numpy(), A.val.cpu().numpy())


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def kernel_name(best, C, inf):
    """The binary64 SpMV kernel the tuned launch runs."""
    long_rows = "true" if inf.max_row_len > 64 else "false"
    if best.pipeline == 2:
        ring = {1: 1, 2: 2, 4: 3, 8: 4}[best.unroll]
        return (f"k_spmv_bulk<double,Plain<double>,{C // 32},{long_rows}> {best.block // 32} warps/block, "
                f"{ring} pieces per warp")
    pipe = 'true' if best.pipeline else 'false'
    if long_rows == "false":  # one vector without long rows: the full-occupancy entry point
        return f"k_spmv_short<double,{best.unroll},{pipe},Plain<double>> block {best.block}"
    return f"k_spmmv<double,1,{best.unroll},{pipe},Plain<double>,true> block {best.block}"


def lookup_traffic(workload_key):
    """dram bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None, None
    e = d.get(workload_key)
    if not e or e.get("src_sha") != kernel_source_hash():
        return None, None
    return e.get("dram_bytes_per_launch"), e.get("note")


# ------------------------------------------------------------------ clocks
class NvmlClocks:
    """The SM clock and the clock-event reasons, polled about once per
    millisecond through NVML (libnvidia-ml; read-only queries), so that even
    a timed region of a few milliseconds carries samples of its own."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, cuda_index):
        self.ok = False
        self.samples = []
        self.max_mhz = None
        self._stop = threading.Event()
        self._thread = None
        try:
            import torch
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return
            dev = ctypes.c_void_p()
            found = False
            try:
                uuid = "GPU-" + str(torch.cuda.get_device_properties(cuda_index).uuid)
                found = lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(dev)) == 0
            except Exception:
                found = False
            if not found and lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(cuda_index), ctypes.byref(dev)) != 0:
                return
            self.lib, self.dev = lib, dev
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(dev, 1, ctypes.byref(mx)) == 0:
                self.max_mhz = float(mx.value)
            self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons", None)
            self.ok = True
        except Exception:
            self.ok = False

    def start(self):
        if self.ok:
            self._thread = threading.Thread(target=self._run, daemon=True)
            self._thread.start()
        return self

    def _run(self):
        clk, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            t = time.perf_counter()
            if self.lib.nvmlDeviceGetClockInfo(self.dev, 1, ctypes.byref(clk)) == 0:
                r = 0
                if self.reasons_fn is not None and self.reasons_fn(self.dev, ctypes.byref(rs)) == 0:
                    r = rs.value
                self.samples.append((t, float(clk.value), r))
            self._stop.wait(0.001)

    def stop(self):
        self._stop.set()
        if self._thread:
            self._thread.join(timeout=2)

    def summary(self, t0, t1):
        """Samples taken between perf_counter() times t0 and t1."""
        if not self.ok:
            return None
        win = [s for s in self.samples if t0 <= s[0] <= t1]
        if not win and self.samples:
            win = [min(self.samples, key=lambda s: abs(s[0] - 0.5 * (t0 + t1)))]
        if not win:
            return None
        reasons = sorted({nm for _, _, r in win for bit, nm in self.REASONS.items() if r & bit})
        return {"sm_mhz": statistics.median(s[1] for s in win), "sm_max_mhz": self.max_mhz,
                "reasons": reasons, "samples": len(win), "source": "nvml, ~1 ms polling"}


class SmiClocks:
    """nvidia-smi sampled every 100 ms over the whole run, summarised per
    section (a window of wall-clock time named by the caller)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.samples = []
        self.proc = None
        self.sections = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return self
        threading.Thread(target=self._read, daemon=True).start()
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.samples.append((time.perf_counter(), [v.strip() for v in ln.split(",")]))

    def section(self, name, t0, t1, note=None):
        self.sections.append((name, t0, t1, note))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        self.proc = None

    def pause(self):
        """Stop sampling for a while (resume() starts a new nvidia-smi)."""
        self.stop()

    def resume(self):
        return self.start()

    def summary(self, t0, t1):
        win = [s for t, s in self.samples if t0 <= t <= t1]
        if not win:
            return {"samples": 0}
        sm = [float(s[1]) for s in win if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in win if s[2].replace(".", "").isdigit()]
        pw = [float(s[3]) for s in win if s[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({nm for s in win for i, nm in enumerate(names)
                          if len(s) > 5 + i and s[5 + i].lower().startswith("active")})
        return {"samples": len(win), "sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "power_w_median": statistics.median(pw) if pw else None}

    def by_section(self):
        out = {}
        for name, t0, t1, note in self.sections:
            out[name] = self.summary(t0, t1)
            if note:
                out[name]["note"] = note
        return out


# ------------------------------------------------------------------ helpers
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def time_spmv(sell, h, xd, yd, stream, reps, warm=3, flags=0):
    import torch
    for _ in range(warm):
        sell.sell_spmv(h, xd, yd, flags=flags, stream=stream)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        sell.sell_spmv(h, xd, yd, flags=flags, stream=stream)
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / reps * 1e-3


def time_spmv_cold(sell, h, xd, yd, stream, reps=50):
    """Average SpMV time with L2 flushed before every call (a 256 MB write
    between calls, outside the timed pair of events)."""
    import torch
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    with torch.cuda.stream(stream):
        for e0, e1 in ev:
            flush.fill_(1)
            e0.record(stream)
            sell.sell_spmv(h, xd, yd, stream=stream)
            e1.record(stream)
    torch.cuda.synchronize()
    t = sum(e0.elapsed_time(e1) for e0, e1 in ev) * 1e-3 / reps
    del flush
    return t


def time_spmmv(sell, h, Xd, Yd, stream, reps, warm=3, flags=0):
    import torch
    for _ in range(warm):
        sell.sell_spmmv(h, Xd, Yd, flags=flags, stream=stream)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        sell.sell_spmmv(h, Xd, Yd, flags=flags, stream=stream)
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / reps * 1e-3


def measure_read_bw(sell, stream, nbytes=4 * 2 ** 30, reps=10):
    """Best-of-reps bandwidth of the read-only kernel (Listing "reduction"
    analogue) over a buffer far larger than L2."""
    import torch
    buf = torch.ones(nbytes // 4, dtype=torch.int32, device="cuda")
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sink = torch.empty(sms * 16, dtype=torch.float64, device="cuda")
    sell.sell_bench_read(buf, nbytes, sink, grid=0, stream=stream)
    best = 1e30
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sell.sell_bench_read(buf, nbytes, sink, grid=0, stream=stream)
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b) * 1e-3)
    del buf
    return nbytes / best / 1e9


def measure_gather(sell, stream, n_words, reps=5, iters=64):
    """Random 8-byte gathers per second from an n_words array (L2-resident
    when n_words * 8 is well below the 129 MB L2)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    grid = sms * 8
    x = torch.ones(n_words, dtype=torch.int64, device="cuda")
    sink = torch.empty(grid * 256, dtype=torch.float64, device="cuda")
    sell.sell_bench_gather(x, n_words, sink, grid, iters, stream=stream)
    best = 1e30
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sell.sell_bench_gather(x, n_words, sink, grid, iters, stream=stream)
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b) * 1e-3)
    return grid * 256 * iters * 8 / best / 1e9


def measure_fp64_fma(sell, stream, iters=6000, clocks=None):
    """Binary64 FMA rate of sell_bench_fma64 over about 0.2 s, and the median
    SM clock sampled meanwhile (a kernel of nothing but FMAs may draw enough
    power to run below the maximum clock; the rate scaled to the maximum
    clock is what an SpMV running at that clock can reach)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    grid = sms * 8
    sink = torch.empty(grid * 256, dtype=torch.float64, device="cuda")
    sell.sell_bench_fma64(sink, grid, 10, stream=stream)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    a.record(stream)
    sell.sell_bench_fma64(sink, grid, iters, stream=stream)
    b.record(stream)
    b.synchronize()
    t1 = time.perf_counter()
    fmas = grid * 256 * iters * 64
    tf = 2.0 * fmas / (a.elapsed_time(b) * 1e-3) / 1e12
    out = {"tflops": round(tf, 4)}
    cs = clocks.summary(t0, t1) if clocks is not None else None
    if cs and cs.get("sm_mhz") and cs.get("sm_max_mhz"):
        out.update({"sm_mhz": cs["sm_mhz"], "sm_max_mhz": cs["sm_max_mhz"], "samples": cs["samples"],
                    "tflops_at_max_clock": round(tf * cs["sm_max_mhz"] / cs["sm_mhz"], 4)})
    return out


def cpu_baseline(A, x, what, target_s=10.0):
    """The oracle's CRS SpMV (binary64, OpenMP on all host cores, STATIC or
    GUIDED,1 by the zeta heuristic of Sec. 5) timed on the full matrix."""
    import oracle
    nth = os.cpu_count() or 1
    zeta = oracle.zeta(A.row_lengths().astype(np.int32))
    guided = zeta >= 0.4
    t0 = time.perf_counter()
    oracle.csr_spmv(A, x, nthreads=nth, guided=guided)
    one = time.perf_counter() - t0
    reps = max(1, int(target_s / max(one, 1e-6)))
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.csr_spmv(A, x, nthreads=nth, guided=guided)
    dt = (time.perf_counter() - t0) / reps
    return {"value": round(2.0 * A.nnz / dt / 1e9, 3), "unit": "GF/s", "cores": nth, "kind": "oracle",
            "sample": f"{what}: the full matrix ({A.nnz} nnz), {reps} calls of the binary64 CRS SpMV, "
                      f"OpenMP {'GUIDED,1' if guided else 'STATIC'} (zeta={zeta:.2f})"}


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle
    from paper_1307_6209_gb300 import synth
    W = workload(args)
    nth = os.cpu_count() or 1
    x = synth.vector(W["nrows"], seed=0)
    budget = 90.0  # seconds for warm-up + timed steps
    calls = args.steps + args.warmup
    if W["name"] == "stencil27":
        # rows of the stencil are generated directly; a probe prefix sizes the sample
        probe = synth.stencil27(round(W["nrows"] ** (1 / 3)), perturb=0.1, seed=0, rows=min(W["nrows"], 200_000))
        zeta = oracle.zeta(probe.row_lengths().astype(np.int32))
        guided = zeta >= 0.4
        oracle.csr_spmv(probe, x, nthreads=nth, guided=guided)
        t0 = time.perf_counter()
        for _ in range(3):
            oracle.csr_spmv(probe, x, nthreads=nth, guided=guided)
        per_row = (time.perf_counter() - t0) / 3 / probe.nrows
        nrow = int(max(1, min(W["nrows"], budget / max(calls * per_row, 1e-12))))
        S = W["host"](nrow)
        total_nnz = W["nnz"]
    else:
        A = W["host"]()
        zeta = oracle.zeta(A.row_lengths().astype(np.int32))
        guided = zeta >= 0.4
        t0 = time.perf_counter()
        oracle.csr_spmv(A, x, nthreads=nth, guided=guided)
        t_full = time.perf_counter() - t0
        frac = min(1.0, budget / max(calls * t_full, 1e-9))
        nrow = max(1, int(A.nrows * frac))
        S = synth.CSR(nrow, A.ncols, A.rpt[:nrow + 1].copy(), A.col[:A.rpt[nrow]], A.val[:A.rpt[nrow]])
        total_nnz = A.nnz
    for _ in range(args.warmup):
        oracle.csr_spmv(S, x, nthreads=nth, guided=guided)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.csr_spmv(S, x, nthreads=nth, guided=guided)
    dt = time.perf_counter() - t0
    gf = 2.0 * S.nnz * args.steps / dt / 1e9
    sample = (f"rows 0..{nrow - 1} of the workload ({S.nnz} nnz, {100 * S.nnz / total_nnz:.2f}% of it) per step, "
              f"binary64 CRS SpMV, OpenMP {'GUIDED,1' if guided else 'STATIC'} on {nth} threads")
    line = {"impl": "reference", "metric": METRIC, "value": round(gf, 3), "unit": "GF/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": W["desc"], "sample": sample},
            "cpu_baseline": {"value": round(gf, 3), "unit": "GF/s", "cores": nth, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(gf, 3), "unit": "GF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def tune_launch(sell, h, xd, yd, stream, flags=0, blocks=(128, 256), unrolls=(1, 2, 4, 8), pipelines=(0, 1, 2)):
    """Pick (block, unroll, pipeline) for one handle: two interleaved timing
    rounds of every candidate, best of the two; returns (block, unroll,
    pipeline, seconds).  Modes the handle does not support are skipped."""
    cands = [(b, u, p) for b in blocks for u in unrolls for p in pipelines]
    best_t = {c: 1e30 for c in cands}
    for _ in range(2):
        for c in cands:
            try:
                sell.sell_set_launch(h, *c)
            except sell.SellError:
                continue
            best_t[c] = min(best_t[c], time_spmv(sell, h, xd, yd, stream, reps=30, flags=flags))
    c, t = min(best_t.items(), key=lambda kv: kv[1])
    sell.sell_set_launch(h, *c)
    return c[0], c[1], c[2], t


def mixed_section(sell, model, csr_d, C, sigma, xd, y64, t64, stream, peak, comps):
    """The same matrix with binary32 and bfloat16 values (binary32 x, y and
    accumulation), each accumulation mode with its own tuned launch; error
    against the binary64 product of the GPU."""
    import torch
    out = {}
    x32 = xd.float()
    nnz = int(csr_d.rpt[-1])
    for name, st in (("f32", sell.SELL_F32), ("bf16", sell.SELL_BF16)):
        hm = sell.sell_build(csr_d, C=C, sigma=sigma, store_type=st, stream=stream)
        inf = hm.info
        y32 = torch.empty(inf.nrows, dtype=torch.float32, device="cuda")
        vb = 4 if st == sell.SELL_F32 else 2
        alg = model.algorithmic_bytes(inf.nrows, inf.ncols, nnz, inf.nchunks, C, vb, 4, inf.has_perm)
        row = {}
        for tag, fl in comps:
            blk, unr, pip, _ = tune_launch(sell, hm, x32, y32, stream, flags=fl)
            dt = time_spmv(sell, hm, x32, y32, stream, reps=100, flags=fl)
            torch.cuda.synchronize()
            err = (y32.double() - y64).abs()
            row[tag] = {"gflops": round(2.0 * nnz / dt / 1e9, 1), "us": round(dt * 1e6, 2),
                        "gbs": round(alg / dt / 1e9, 1), "hbm_frac": round(alg / dt / 1e9 / peak, 4),
                        "speedup_vs_f64": round(t64 / dt, 3), "block": blk, "unroll": unr, "pipeline": pip,
                        "max_abs_err_vs_f64": float(err.max()), "rel_err_vs_f64": float(err.norm() / y64.norm())}
        out[name] = row
        hm.free()
    return out


def lognormal_section(sell, autotune, model, stream, peak, gather_gps, fma_tf):
    """The lognormal random matrix, N = 2,000,000 (irregular, random columns):
    the C x sigma sweep of the paper's Sec. 5.3 with the autotuner's choice,
    its HBM and L2-gather bounds, cold calls, SpMMV and reduced precision."""
    import torch
    from paper_1307_6209_gb300 import synth
    n = 2_000_000
    A = synth.lognormal(n, mean=16.0, sigma_ln=1.2, cap=2000, seed=0)
    csr_d = to_device(A)
    x = torch.from_numpy(synth.vector(n, seed=0)).cuda()
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    tr = autotune.tune(csr_d, store_type=sell.SELL_F64, Cs=(32, 64, 128), sigmas=(1, 256, 4096, n),
                       blocks=(128, 256, 512), unrolls=(1, 2, 4, 8), pipelines=(0, 1, 2), keep=2, stream=stream,
                       use_cache=False, cache=None)
    best = tr.best
    h = autotune.build_tuned(csr_d, best, stream=stream)
    inf = h.info
    dt = time_spmv(sell, h, x, y, stream, reps=500)
    alg = model.algorithmic_bytes(n, n, A.nnz, inf.nchunks, best.C, 8, 8, inf.has_perm)
    out = {"workload": f"lognormal random N={n} (row length mean 16, log-sd 1.2, cap 2000), nnz={A.nnz}, FP64",
           "nnz": A.nnz, "tuned": {"C": best.C, "sigma": best.sigma, "block": best.block, "unroll": best.unroll,
                                   "pipeline": best.pipeline},
           "beta": round(inf.beta, 6), "zeta": round(inf.zeta, 3),
           "us": round(dt * 1e6, 2), "gflops": round(2.0 * A.nnz / dt / 1e9, 1),
           "gbs": round(alg / dt / 1e9, 1), "hbm_frac": round(alg / dt / 1e9 / peak, 4),
           "kernel": kernel_name(best, best.C, inf),
           "gather_bound": {"achieved_ggps": round(A.nnz / dt / 1e9, 1), "peak_ggps_measured": round(gather_gps, 1),
                            "frac": round(A.nnz / dt / 1e9 / gather_gps, 4),
                            "bound_us": round(A.nnz / gather_gps / 1e3, 2)},
           "fp64_pipe_frac": round(2.0 * A.nnz / dt / 1e12 / fma_tf, 4),
           "sweep": [{"C": f["C"], "sigma": f["sigma"], "beta": round(f["beta"], 4), "us": round(f["us"], 2),
                      "gflops": round(2.0 * A.nnz / f["us"] / 1e3, 1), "build_ms": round(f["build_ms"], 2)}
                     for f in sorted(tr.formats, key=lambda f: (f["C"], f["sigma"]))]}
    nnzr = A.nnz / n
    bal = model.balance_sell(1.0 / nnzr, inf.beta, nnzr)
    out["paper_model"] = {"balance_bytes_per_flop": round(bal, 4),
                          "model_bytes_per_launch": int(model.paper_model_bytes(A.nnz, inf.beta, n, n))}
    cold = time_spmv_cold(sell, h, x, y, stream)
    out["cold_us"] = round(cold * 1e6, 2)
    spmmv = {}
    for k in (4, 8):
        Xd = x[:, None].repeat(1, k).contiguous()
        Yd = torch.empty((n, k), dtype=torch.float64, device="cuda")
        t = time_spmmv(sell, h, Xd, Yd, stream, reps=50)
        spmmv[f"k{k}"] = {"gflops": round(2.0 * A.nnz * k / t / 1e9, 1), "us": round(t * 1e6, 2)}
        del Xd, Yd
    out["spmmv_f64"] = spmmv
    sell.sell_spmv(h, x, y, stream=stream)
    torch.cuda.synchronize()
    out["mixed"] = mixed_section(sell, model, csr_d, best.C, best.sigma, x, y.clone(), dt, stream, peak,
                                 (("plain", 0), ("dot2", sell.SELL_SPMV_COMPENSATED),
                                  ("dot2_long_rows", sell.SELL_SPMV_COMPENSATED_LONG)))
    h.free()
    del csr_d, A
    torch.cuda.empty_cache()
    return out


def laplace_section(sell, stream, reps=2000):
    """The 5-point Laplacian on 64 x 64 (N = 4096, 20,224 nnz), SELL-32-1: an
    L2-resident product bound by launch latency, so the number is the time
    per call, back to back on one stream and inside one CUDA graph."""
    import torch
    from paper_1307_6209_gb300 import synth
    A = synth.laplace2d(64)
    h = sell.sell_build(A, C=32, sigma=1, stream=stream)
    x = torch.from_numpy(synth.vector(A.ncols, seed=0)).cuda()
    y = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
    eager = time_spmv(sell, h, x, y, stream, reps=reps)
    g = torch.cuda.CUDAGraph()
    per_graph = 100
    with torch.cuda.stream(stream):
        sell.sell_spmv(h, x, y, stream=stream)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=stream):
            for _ in range(per_graph):
                sell.sell_spmv(h, x, y, stream=torch.cuda.current_stream())
        g.replay()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps // per_graph):
            g.replay()
        b.record(stream)
        b.synchronize()
    graph = a.elapsed_time(b) * 1e-3 / (reps // per_graph * per_graph)
    h.free()
    return {"workload": "5-point Laplacian 64x64, N=4096, nnz=20224, SELL-32-1", "us_per_call": round(eager * 1e6, 2),
            "us_per_call_in_graph": round(graph * 1e6, 2), "gflops": round(2.0 * A.nnz / eager / 1e9, 2)}


def _time_graph(g, stream, reps):
    """Average time of one replay; the replays run on `stream`, where the
    events are recorded (a graph replays on the current stream)."""
    import torch
    with torch.cuda.stream(stream):
        g.replay()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            g.replay()
        b.record(stream)
        b.synchronize()
    return a.elapsed_time(b) * 1e-3 / reps


def batched_section(sell, autotune, model, stream, peak, gather_gps, nmat=512, ks=(1, 4, 8), seed=0):
    """512 matrices, rows U[1k, 200k], half banded (bandwidth 64, 7-30 per
    row), half lognormal; FP32 storage; k right-hand sides; C and sigma tuned
    per class.  One plan per k (CUDA graph) against per-matrix launches and
    against the same batch in FP64.  Every product of the plan is checked
    bitwise against the same product alone."""
    import torch
    from paper_1307_6209_gb300 import synth
    gen = {"banded": synth.banded_device, "lognormal": synth.lognormal_device}
    recipe = synth.batch_set(nmat, seed=seed)
    rng = np.random.default_rng(seed + 1)
    # C and sigma per class, tuned for batch throughput on 16 sample matrices
    # (a single small matrix is latency-bound and would favour formats that
    # move more bytes)
    choice = {}
    for cls in ("banded", "lognormal"):
        samples = [gen[cls](int(n), seed=900 + j) for j, n in enumerate(rng.integers(1000, 200001, 16))]
        best, table = autotune.tune_batch(samples, store_type=sell.SELL_F32, stream=stream)
        choice[cls] = {"C": best["C"], "sigma": best["sigma"],
                       "candidates": [{k: (round(v, 1) if k == "us" else v) for k, v in t.items()} for t in table]}
        del samples
    h32, h64, kinds, nnz = [], [], [], 0
    t0 = time.perf_counter()
    for kind, n, s in recipe:
        A = gen[kind](n, seed=s)
        ch = choice[kind]
        h32.append(sell.sell_build(A, C=ch["C"], sigma=ch["sigma"], store_type=sell.SELL_F32, stream=stream))
        h64.append(sell.sell_build(A, C=ch["C"], sigma=ch["sigma"], store_type=sell.SELL_F64, stream=stream))
        kinds.append(kind)
        nnz += A.nnz
        del A
    build_s = time.perf_counter() - t0
    out = {"workload": f"{nmat} matrices, rows U[1000, 200000], half banded (bw 64, 7-30/row), half lognormal",
           "nnz_total": nnz, "rows_total": int(sum(n for _, n, _ in recipe)),
           "tuned": {c: {"C": v["C"], "sigma": v["sigma"]} for c, v in choice.items()},
           "tuning_candidates": {c: v["candidates"] for c, v in choice.items()},
           "build_s_both_precisions": round(build_s, 2)}
    for k in ks:
        row = {}
        for tag, hs, dt, vb in (("f32", h32, torch.float32, 4), ("f64", h64, torch.float64, 8)):
            items = []
            for h in hs:
                shp_x = (h.info.ncols,) if k == 1 else (h.info.ncols, k)
                shp_y = (h.info.nrows,) if k == 1 else (h.info.nrows, k)
                items.append((h, torch.rand(shp_x, dtype=dt, device="cuda"),
                              torch.empty(shp_y, dtype=dt, device="cuda"), 0))
            # the plan's launch (rows per block, right-hand-side block width)
            # tuned on the plan itself; it changes no result
            lt, ltable = autotune.tune_plan(items, k, stream=stream)
            rflag = {8: 0, 4: sell.SELL_SPMV_RHS_BLOCK4}[lt["rhs"]]
            items = [(h, X, Y, rflag) for h, X, Y, _ in items]
            plan = sell.sell_batch_create(items, stream=stream)
            plan.set_launch(lt["tile"])
            plan.run(stream=stream)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                plan.run(stream=stream)
            t_batch = _time_graph(g, stream, 20)
            batch_y = [Y.clone() for _, _, Y, _ in items]

            def per_matrix():
                for h, X, Y, fl in items:
                    if k == 1:
                        sell.sell_spmv(h, X, Y, stream=stream)
                    else:
                        sell.sell_spmmv(h, X, Y, flags=fl, stream=stream)
            per_matrix()
            torch.cuda.synchronize()
            same = all(torch.equal(a, Y) for a, (_, _, Y, _) in zip(batch_y, items))
            del batch_y
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(3):
                per_matrix()
            b.record(stream)
            b.synchronize()
            t_eager = a.elapsed_time(b) * 1e-3 / 3
            g2 = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g2, stream=stream):
                per_matrix()
            t_pm_graph = _time_graph(g2, stream, 5)
            # bound weighted by class: the banded products at the HBM copy
            # bandwidth, the lognormal ones (random columns) at the measured
            # L2 gather rate (or HBM, whichever is slower)
            alg = {"banded": 0, "lognormal": 0}
            gath = 0
            for h, kind in zip(hs, kinds):
                inf = h.info
                alg[kind] += model.algorithmic_bytes(inf.nrows, inf.ncols, inf.nnz, inf.nchunks, inf.C, vb, vb,
                                                     inf.has_perm, k=k)
                gath += inf.nnz if kind == "lognormal" else 0
            t_bound = alg["banded"] / (peak * 1e9) + max(alg["lognormal"] / (peak * 1e9), gath / (gather_gps * 1e9))
            row[tag] = {"batch_ms": round(t_batch * 1e3, 3), "gflops": round(2.0 * nnz * k / t_batch / 1e9, 1),
                        "tuned_launch": {"block": lt["tile"], "rhs_block": lt["rhs"]},
                        "launch_candidates": [{"block": c["tile"], "rhs_block": c["rhs"], "us": round(c["us"], 1)}
                                              for c in ltable],
                        "hbm_frac": round((alg["banded"] + alg["lognormal"]) / t_batch / 1e9 / peak, 4),
                        "class_bound_ms": round(t_bound * 1e3, 3), "class_bound_frac": round(t_bound / t_batch, 4),
                        "per_matrix_eager_ms": round(t_eager * 1e3, 3),
                        "per_matrix_graph_ms": round(t_pm_graph * 1e3, 3),
                        "speedup_vs_per_matrix_eager": round(t_eager / t_batch, 2),
                        "speedup_vs_per_matrix_graph": round(t_pm_graph / t_batch, 2),
                        "batch_equals_per_matrix": same}
            plan.free()
            del g, g2, items
        row["f32_speedup_vs_f64"] = round(row["f64"]["batch_ms"] / row["f32"]["batch_ms"], 3)
        out[f"k{k}"] = row
    # the banded half alone (regular, memory-bound matrices), binary32, k = 1
    hb = [h for h, kind in zip(h32, kinds) if kind == "banded"]
    items = [(h, torch.rand(h.info.ncols, dtype=torch.float32, device="cuda"),
              torch.empty(h.info.nrows, dtype=torch.float32, device="cuda"), 0) for h in hb]
    lt, _ = autotune.tune_plan(items, 1, stream=stream)
    plan = sell.sell_batch_create(items, stream=stream)
    plan.set_launch(lt["tile"])
    plan.run(stream=stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        plan.run(stream=stream)
    t_b = _time_graph(g, stream, 20)
    alg_b = sum(model.algorithmic_bytes(h.info.nrows, h.info.ncols, h.info.nnz, h.info.nchunks, h.info.C, 4, 4,
                                        h.info.has_perm) for h in hb)
    nnz_b = sum(h.info.nnz for h in hb)
    out["banded_only_f32_k1"] = {"matrices": len(hb), "nnz": nnz_b, "batch_ms": round(t_b * 1e3, 3),
                                 "gflops": round(2.0 * nnz_b / t_b / 1e9, 1),
                                 "hbm_frac": round(alg_b / t_b / 1e9 / peak, 4), "block": lt["tile"]}
    plan.free()
    del g, items
    for h in h32 + h64:
        h.free()
    torch.cuda.empty_cache()
    return out


def serving_section(sell, stream, nmat=64, seed=0, duration_s=1.5, repeats=3):
    """64 resident matrices, rows log-uniform in [10k, 4M], lognormal row
    lengths, half FP64 and half FP32; requests of 1-8 right-hand sides from
    pinned host memory; Poisson arrivals at fractions of the saturated rate,
    each load three times (seeds 7, 8, 9) for the run-to-run spread; latency
    percentiles overall and per size class (small: work at most the median
    request's), the worst latency per 50 ms of arrivals (the tail's timing),
    and one request alone."""
    import torch
    from paper_1307_6209_gb300 import serving, synth
    rng = np.random.default_rng(seed)
    rows = np.exp(rng.uniform(np.log(10_000), np.log(4_000_000), nmat)).astype(np.int64)
    mats = []
    for i, n in enumerate(rows):
        A = synth.lognormal_device(int(n), seed=1000 + i)
        st = sell.SELL_F64 if i % 2 == 0 else sell.SELL_F32
        mats.append(sell.sell_build(A, C=32, sigma=int(n), store_type=st, stream=stream))
        del A
    resident = sum(h.info.device_bytes for h in mats)
    budget = resident + (8 << 30)
    # one pinned input buffer per matrix (room for 8 right-hand sides); a
    # request of k columns uses its first ncols * k elements (inputs are
    # read-only, so concurrent requests may share them)
    pool = []
    for h in mats:
        dt = torch.float64 if h.info.store_type == sell.SELL_F64 else torch.float32
        pool.append((torch.rand(h.info.ncols * 8, dtype=dt) * 2 - 1).pin_memory())

    def make(g):
        mid = int(g.integers(0, nmat))
        k = int(g.integers(1, 9))
        n = mats[mid].info.ncols
        buf = pool[mid]
        return mid, (buf[:n] if k == 1 else buf[:n * k].view(n, k))

    works = sorted(int(h.info.stored) * k for h in mats for k in range(1, 9))
    small_work = works[len(works) // 2]

    def one_load(rate, sd):
        srv = serving.Server(mats, budget, max_batch=64, streams=6)
        reqs = serving.poisson_load(srv, rate_hz=rate, duration_s=duration_s, make_request=make, seed=sd,
                                    to_host=False)
        t_end = max(r.t_done for r in reqs)
        t_beg = min(r.t_arrive for r in reqs)
        st = srv.stats(split_work=small_work)
        srv.stop()
        gfl = sum(2.0 * mats[r.mid].info.nnz * r.k for r in reqs)
        st["throughput_req_per_s"] = len(reqs) / (t_end - t_beg)
        st["gflops"] = gfl / (t_end - t_beg) / 1e9
        lat = np.array([r.t_done - r.t_arrive for r in reqs]) * 1e3
        wait = np.array([r.t_launch - r.t_arrive for r in reqs]) * 1e3
        st["wait_p99_ms"] = float(np.percentile(wait, 99))
        bins = ((np.array([r.t_arrive for r in reqs]) - t_beg) / 0.05).astype(int)
        st["worst_ms_per_50ms"] = [round(float(lat[bins == b].max()), 1) if (bins == b).any() else 0.0
                                   for b in range(int(bins.max()) + 1)]
        return st

    def rnd(d):
        return {k: (rnd(v) if isinstance(v, dict) else round(v, 3) if isinstance(v, float) else v) for k, v in d.items()}

    out = {"workload": f"{nmat} resident matrices, rows log-uniform [10k, 4M], lognormal rows, half FP64 / "
                       f"half FP32, requests k ~ U{{1..8}}, inputs from pinned host memory, results left on "
                       f"the device and taken by a client thread as they complete; latency = arrival to the "
                       f"batch's completion; scheduler, admission and batching in the native server "
                       f"(6 streams, batches of up to 64)",
           "resident_gb": round(resident / 1e9, 2), "budget_gb": round(budget / 1e9, 2),
           "nnz_total": int(sum(h.info.nnz for h in mats)),
           "small_request_work": small_work,
           "size_classes": "small: stored elements x k at most the median request's; large: the rest"}
    # warm-up (kernels, arena, pinned memory); three bursts of 400 requests
    # for context (one burst lasts ~50 ms, so a single stall halves its rate);
    # then the saturated rate: completions per second in steady state, 256
    # requests kept outstanding for 2 s
    srv = serving.Server(mats, budget, max_batch=64, streams=6)
    serving.burst_load(srv, 200, make, seed=1, to_host=False)
    srv.stop()
    sats = []
    for sd in (2, 3, 4):
        srv = serving.Server(mats, budget, max_batch=64, streams=6)
        burst, dt = serving.burst_load(srv, 400, make, seed=sd, to_host=False)
        sats.append(len(burst) / dt)
        if sd == 2:
            out["burst"] = rnd(srv.stats(split_work=small_work))
        srv.stop()
    out["burst_req_per_s"] = [round(v, 1) for v in sats]
    srv = serving.Server(mats, budget, max_batch=64, streams=6)
    n_done, dt = serving.closed_loop(srv, 256, 2.0, make, seed=5, to_host=False)
    st = srv.stats()
    srv.stop()
    # (the burst median stands in if the closed loop completed nothing)
    sat = n_done / dt if n_done > 0 and dt > 0 else statistics.median(sats)
    out["saturated_req_per_s"] = round(sat, 1)
    out["saturated_how"] = "closed loop, 256 requests outstanding, 2 s"
    out["saturated_mean_batch"] = round(st["mean_batch"], 2)
    for frac in (0.5, 0.8, 0.95):
        runs = [one_load(frac * sat, 7 + rep) for rep in range(repeats)]
        row = rnd(runs[0])
        row["offered_req_per_s"] = round(frac * sat, 1)
        for key in ("p50_ms", "p99_ms", "wait_p99_ms", "throughput_req_per_s"):
            vals = [r[key] for r in runs]
            row[key] = round(statistics.median(vals), 3)
            row[key + "_runs"] = [round(v, 3) for v in vals]
        for cls in ("small", "large"):
            if all(cls in r for r in runs):
                row[cls] = {key: round(statistics.median(r[cls][key] for r in runs), 3) for key in ("p50_ms", "p99_ms")}
                row[cls]["requests"] = runs[0][cls]["requests"]
        out[f"load_{frac}"] = row
    # one request alone: the largest request (the 4M-row matrix, k = 8) and
    # a small one, each through the server on an idle GPU
    srv = serving.Server(mats, budget, max_batch=64, streams=2)
    big = int(np.argmax([h.info.stored for h in mats]))
    little = int(np.argmin([h.info.stored for h in mats]))
    alone = {}
    for tag, mid, k in (("largest_k8", big, 8), ("smallest_k1", little, 1)):
        lat = []
        for _ in range(5):
            n = mats[mid].info.ncols
            X = pool[mid][:n] if k == 1 else pool[mid][:n * k].view(n, k)
            r = srv.submit(mid, X, to_host=False)
            r.wait(60)
            lat.append(r.latency * 1e3)
            r.release()
        alone[tag] = round(statistics.median(lat), 3)
    srv.stop()
    out["alone_ms"] = alone
    for h in mats:
        h.free()
    torch.cuda.empty_cache()
    return out


def serving_in_subprocess(timeout_s=900):
    """The serving section in a process of its own (`bench.py --section
    serving`), so that the latency it measures is not shaped by the state the
    other sections leave in this one (threads, memory pools, handles)."""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--section", "serving"], capture_output=True,
                       text=True, timeout=timeout_s, cwd=ROOT)
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    if r.returncode != 0 or not lines:
        raise RuntimeError(f"serving subprocess rc={r.returncode}: {r.stderr[-400:]}")
    out = json.loads(lines[-1])
    out["process"] = "own process (bench.py --section serving)"
    return out


def run_section(args):
    import torch
    from paper_1307_6209_gb300 import build as cuda_build
    from paper_1307_6209_gb300 import sell
    _, _, local = dist_setup()
    torch.cuda.set_device(local)
    cuda_build.build()
    sell.load()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        out = serving_section(sell, stream)
    print(json.dumps(out), flush=True)
    return 0


def pathological_section(sell, model, stream, peak):
    """The shapes Sec. 5.2 singles out for accelerators: a dense 8000 x 8000
    matrix stored as sparse (few rows, long rows; the paper quotes 7.3 / 23 /
    17 GF/s on SNB / Phi / K20 and 31 GF/s on K20 with 16 threads per row) and
    a webbase-1M-like matrix (1M rows of 3 entries plus one row of 1M)."""
    import torch
    from paper_1307_6209_gb300 import synth
    out = {}
    cases = (("dense8000", lambda: synth.dense_device(8000), ((32, 1),)),
             ("webbase_like_1M", lambda: synth.long_row_device(1_000_000, 1_000_000, short_len=3, at=12345),
              ((32, 1), (32, 1 << 30))))
    for name, make, fmts in cases:
        A = make()
        x = torch.rand(A.ncols, dtype=torch.float64, device="cuda")
        y = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
        for C, sg in fmts:
            h = sell.sell_build(A, C=C, sigma=sg, stream=stream)
            blk, unr, pip, _ = tune_launch(sell, h, x, y, stream)
            dt = time_spmv(sell, h, x, y, stream, reps=50)
            alg = model.algorithmic_bytes(A.nrows, A.ncols, A.nnz, h.info.nchunks, C, 8, 8, h.info.has_perm)
            out[f"{name}_C{C}_s{sg}"] = {"nnz": A.nnz, "us": round(dt * 1e6, 2),
                                          "gflops": round(2.0 * A.nnz / dt / 1e9, 1),
                                          "hbm_frac": round(alg / dt / 1e9 / peak, 4), "beta": round(h.info.beta, 4),
                                          "block": blk, "unroll": unr, "pipeline": pip}
            h.free()
        del A, x, y
        torch.cuda.empty_cache()
    return out


def compact_summary(line, ex):
    """Every figure of the line in a few hundred bytes (placed last, so a
    truncated tail of the output still shows it)."""
    def g(d, *path):
        for p in path:
            if not isinstance(d, dict) or p not in d:
                return None
            d = d[p]
        return d

    s = {"headline": {"gf": line["value"], "hbm": line["roofline"]["frac"], "us": line["roofline"]["kernel_avg_us"],
                      "e2e_gf": g(line, "e2e", "value")}}
    for tag in ("f32", "bf16"):
        r = g(ex, "mixed", tag, "plain")
        if r:
            s[f"headline_{tag}"] = {"gf": r["gflops"], "hbm": r["hbm_frac"], "x_f64": r["speedup_vs_f64"],
                                    "rel_err": float(f"{r['rel_err_vs_f64']:.2e}")}
    ln = ex.get("lognormal2M")
    if isinstance(ln, dict) and "gflops" in ln:
        s["lognormal2M"] = {"gf": ln["gflops"], "hbm": ln["hbm_frac"], "gather": ln["gather_bound"]["frac"],
                            "C": ln["tuned"]["C"], "sigma": ln["tuned"]["sigma"]}
        for tag in ("f32", "bf16"):
            r = g(ln, "mixed", tag, "plain")
            if r:
                s[f"lognormal2M_{tag}"] = {"gf": r["gflops"], "x_f64": r["speedup_vs_f64"],
                                           "rel_err": float(f"{r['rel_err_vs_f64']:.2e}")}
    b = ex.get("batched")
    if isinstance(b, dict) and "k1" in b:
        s["batch512_f32"] = {f"k{k}": {"gf": g(b, f"k{k}", "f32", "gflops"), "hbm": g(b, f"k{k}", "f32", "hbm_frac"),
                                       "bound": g(b, f"k{k}", "f32", "class_bound_frac"),
                                       "x_f64": g(b, f"k{k}", "f32_speedup_vs_f64"),
                                       "ok": g(b, f"k{k}", "f32", "batch_equals_per_matrix")} for k in (1, 4, 8)}
        s["batch512_f32"]["banded_only_k1_hbm"] = g(b, "banded_only_f32_k1", "hbm_frac")
    v = ex.get("serving")
    if isinstance(v, dict) and "load_0.5" in v:
        s["serving"] = {"sat_rps": v["saturated_req_per_s"]}
        for f in ("0.5", "0.8", "0.95"):
            s["serving"][f"p50_p99_ms_{f}"] = [g(v, f"load_{f}", "p50_ms"), g(v, f"load_{f}", "p99_ms")]
        s["serving"]["p99_runs_0.8"] = g(v, "load_0.8", "p99_ms_runs")
        s["serving"]["small_p50_p99_ms_0.8"] = [g(v, "load_0.8", "small", "p50_ms"), g(v, "load_0.8", "small", "p99_ms")]
        s["serving"]["alone_ms"] = v.get("alone_ms")
    lp = ex.get("laplace64")
    if isinstance(lp, dict) and "us_per_call" in lp:
        s["laplace64_us"] = [lp["us_per_call"], lp["us_per_call_in_graph"]]
    errs = [k for k, v in ex.items() if isinstance(v, dict) and "error" in v]
    if errs:
        s["section_errors"] = errs
    return s


def run_ours(args):
    import torch
    from paper_1307_6209_gb300 import autotune
    from paper_1307_6209_gb300 import build as cuda_build
    from paper_1307_6209_gb300 import dist as sdist
    from paper_1307_6209_gb300 import model, sell, synth

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    cuda_build.build()
    sell.load()
    stream = torch.cuda.Stream()
    W = workload(args)
    n_gpus = ws
    dev_name = torch.cuda.get_device_name(local)
    peak, peak_src = load_peaks()
    smi = SmiClocks(local).start()
    nvml = NvmlClocks(local).start()
    extras = {}

    with torch.cuda.stream(stream):
        t_sec = time.perf_counter()
        A_host = None
        if W["device"] is not None:
            csr_d = W["device"]()
        else:
            A_host = W["host"]()
            csr_d = to_device(A_host)
        nrows, ncols, nnz = int(csr_d.nrows), int(csr_d.ncols), int(csr_d.rpt[-1])
        x = synth.vector(ncols, seed=0)
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty(nrows, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()

        # ---- measuring kernels: read bandwidth b, random-gather rate, FP64 FMA peak
        b_read = measure_read_bw(sell, stream)
        gather_gps = measure_gather(sell, stream, 2_000_000)
        fma = measure_fp64_fma(sell, stream, clocks=nvml)
        fma_tf = fma.get("tflops_at_max_clock", fma["tflops"])

        # ---- autotuner: stage 1 = the (C, sigma) candidates, stage 2 = launch shapes
        if args.C is not None or args.sigma is not None or args.no_sweep:
            Cs, sigmas = (args.C or 32,), (args.sigma or 1,)
        else:
            Cs, sigmas = sorted({c for c, _ in W["grid"]}), sorted({s for _, s in W["grid"]})
        blocks = (args.block,) if args.block else (128, 256, 512)
        unrolls = (args.unroll,) if args.unroll else (1, 2, 4, 8)
        pipelines = (args.pipeline,) if args.pipeline is not None else (0, 1, 2)
        tr = autotune.tune(csr_d, store_type=sell.SELL_F64, Cs=Cs, sigmas=sigmas, blocks=blocks,
                           unrolls=unrolls, pipelines=pipelines, keep=2, stream=stream, use_cache=False,
                           cache=None)
        best = tr.best
        C, sigma = best.C, best.sigma
        t0 = time.perf_counter()
        h = autotune.build_tuned(csr_d, best, stream=stream)
        build_ms = (time.perf_counter() - t0) * 1e3
        inf = h.info
        sweep = [{"C": f["C"], "sigma": f["sigma"], "beta": round(f["beta"], 4), "us": round(f["us"], 2),
                  "gflops": round(2.0 * nnz / f["us"] / 1e3, 1), "build_ms": round(f["build_ms"], 2)}
                 for f in sorted(tr.formats, key=lambda f: (f["C"], f["sigma"]))]
        smi.section("setup_and_tuning", t_sec, time.perf_counter())

        # ---- the timed region: K steps of one SpMV each
        for _ in range(args.warmup):
            sell.sell_spmv(h, xd, yd, stream=stream)
        ev_a = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ev_b = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        pc0 = time.perf_counter()
        torch.cuda.nvtx.range_push("timed_region")
        t_start.record(stream)
        for i in range(args.steps):
            ev_a[i].record(stream)
            sell.sell_spmv(h, xd, yd, stream=stream)
            ev_b[i].record(stream)
        t_end.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        pc1 = time.perf_counter()
        if dist:
            dist.barrier()
        smi.section("timed_region", pc0, pc1)
        total_s = t_start.elapsed_time(t_end) * 1e-3
        kern_s = sum(a.elapsed_time(b) for a, b in zip(ev_a, ev_b)) * 1e-3 / args.steps
        flops = 2.0 * nnz
        # weak scaling: every rank's flops over the slowest rank's time
        value = sdist.weak_scaling_throughput(flops * args.steps, total_s, device="cuda") / 1e9
        step_s = sdist.max_over_ranks(total_s, device="cuda") / args.steps
        clocks = nvml.summary(pc0, pc1) or smi.summary(pc0, pc1)

        # ---- the same product back to back for about a second: the clock
        # under sustained load next to the rate it gives
        reps = max(1, int(1.0 / max(kern_s, 1e-6)))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pcs0 = time.perf_counter()
        a.record(stream)
        for _ in range(reps):
            sell.sell_spmv(h, xd, yd, stream=stream)
        b.record(stream)
        b.synchronize()
        pcs1 = time.perf_counter()
        smi.section("sustained", pcs0, pcs1)
        sus_s = a.elapsed_time(b) * 1e-3 / reps
        extras["sustained"] = {"calls": reps, "gflops": round(flops / sus_s / 1e9, 2), "us": round(sus_s * 1e6, 2),
                               "clocks": nvml.summary(pcs0, pcs1) or smi.summary(pcs0, pcs1)}
        nvml.stop()  # the 1 kHz polling thread is for the timed region only

        e2e = None
        if True:  # the end-to-end rate belongs to the line in every mode
            # ---- end to end through the C ABI with host buffers (pinned): each
            # step copies its x in and its y out; steps rotate over NS streams
            # (and NS pinned buffer pairs), so a step's copies overlap the
            # kernels of the steps before it and no input copy waits in its
            # stream behind a result copy it does not need -- the library
            # orders the kernels
            t_sec = time.perf_counter()
            NS = 4
            xh = [torch.from_numpy(x).pin_memory() for _ in range(NS)]
            yh = [torch.empty(nrows, dtype=torch.float64).pin_memory() for _ in range(NS)]
            io_streams = [stream] + [torch.cuda.Stream() for _ in range(NS - 1)]
            ke = min(max(args.steps, 20), 2000)
            for i in range(2 * NS):
                sell.sell_spmv(h, xh[i % NS], yh[i % NS], flags=sell.SELL_SPMV_HOST_IO, stream=io_streams[i % NS])
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(io_streams[0])
            for s_ in io_streams[1:]:
                s_.wait_event(a)
            for i in range(ke):
                sell.sell_spmv(h, xh[i % NS], yh[i % NS], flags=sell.SELL_SPMV_HOST_IO, stream=io_streams[i % NS])
            for s_ in io_streams[1:]:
                io_streams[0].wait_stream(s_)
            b.record(io_streams[0])
            b.synchronize()
            e2e_s = a.elapsed_time(b) * 1e-3 / ke
            e2e_check = all(np.array_equal(yh[0].numpy(), y_.numpy()) for y_ in yh[1:]) and \
                yh[0].numpy().tobytes() == yd.cpu().numpy().tobytes()
            staged = {"gflops": round(n_gpus * flops / e2e_s / 1e9, 2), "ms_per_step": round(e2e_s * 1e3, 4),
                      "result_equals_device_run": e2e_check,
                      "how": f"SELL_SPMV_HOST_IO: x copied in and y out through staging slots, steps rotating "
                             f"over {NS} streams"}
            # the same steps with the kernels reading x from and writing y to
            # the pinned host buffers in place (SELL_SPMV_HOST_DIRECT)
            for i in range(6):
                sell.sell_spmv(h, xh[i % 2], yh[i % 2], flags=sell.SELL_SPMV_HOST_DIRECT, stream=stream)
            torch.cuda.synchronize()
            yh[0].fill_(float("nan"))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for i in range(min(ke, 200)):
                sell.sell_spmv(h, xh[i % 2], yh[i % 2], flags=sell.SELL_SPMV_HOST_DIRECT, stream=stream)
            b.record(stream)
            b.synchronize()
            d_s = a.elapsed_time(b) * 1e-3 / min(ke, 200)
            d_check = yh[0].numpy().tobytes() == yd.cpu().numpy().tobytes()
            direct = {"gflops": round(n_gpus * flops / d_s / 1e9, 2), "ms_per_step": round(d_s * 1e3, 4),
                      "result_equals_device_run": d_check,
                      "how": "SELL_SPMV_HOST_DIRECT: the kernel reads x from and writes y to the pinned host "
                             "buffers over the host link"}
            best_e2e, mode = max(((staged["gflops"], "host_io"), (direct["gflops"] if d_check else 0.0,
                                                                  "host_direct")))
            e2e = {"value": best_e2e, "unit": "GF/s", "h2d_bytes_per_step": 8 * ncols, "d2h_bytes_per_step": 8 * nrows,
                   "steps": ke, "mode": mode, "host_io": staged, "host_direct": direct,
                   "result_equals_device_run": e2e_check and (d_check or mode == "host_io")}
            del xh, yh
            smi.section("e2e", t_sec, time.perf_counter())

        if not args.no_extras:
            # ---- multiple right-hand sides (A streamed once for k vectors)
            t_sec = time.perf_counter()
            spmmv = {}
            for k in (4, 8):
                Xd = xd[:, None].repeat(1, k).contiguous()
                Yd = torch.empty((nrows, k), dtype=torch.float64, device="cuda")
                dt = time_spmmv(sell, h, Xd, Yd, stream, reps=20)
                spmmv[f"k{k}"] = {"gflops": round(2.0 * nnz * k / dt / 1e9, 1), "us": round(dt * 1e6, 2)}
                del Xd, Yd
            extras["spmmv_f64"] = spmmv

            # ---- cold: L2 flushed before each call
            cold_s = time_spmv_cold(sell, h, xd, yd, stream)
            extras["cold"] = {"us": round(cold_s * 1e6, 2), "gflops": round(flops / cold_s / 1e9, 1),
                              "warm_us": round(kern_s * 1e6, 2), "note": "256 MB written between calls"}

            # ---- FP64 vs mixed: binary32 / bfloat16 values, binary32 accumulation
            sell.sell_spmv(h, xd, yd, stream=stream)
            torch.cuda.synchronize()
            comps = [("plain", 0), ("dot2", sell.SELL_SPMV_COMPENSATED)]
            if inf.max_row_len > 64:
                comps.append(("dot2_long_rows", sell.SELL_SPMV_COMPENSATED_LONG))
            extras["mixed"] = mixed_section(sell, model, csr_d, C, sigma, xd, yd.clone(), kern_s, stream, peak,
                                            comps)
            smi.section("spmmv_cold_mixed", t_sec, time.perf_counter())
        if A_host is None and rank == 0 and ws == 1 and not args.no_cpu:
            A_host = to_host(csr_d)  # the matrix the GPU multiplied, for the CPU baseline
        del csr_d
        h.free()
        torch.cuda.empty_cache()
        if not args.no_extras and rank == 0:
            # each extra section reports its own failure instead of losing the line
            sections = [("lognormal2M", lambda: lognormal_section(sell, autotune, model, stream, peak, gather_gps,
                                                                  fma_tf)),
                        ("laplace64", lambda: laplace_section(sell, stream)),
                        ("pathological", lambda: pathological_section(sell, model, stream, peak)),
                        ("batched", lambda: batched_section(sell, autotune, model, stream, peak, gather_gps)),
                        ("serving", lambda: serving_in_subprocess())]
            if W["name"] == "lognormal":
                sections = sections[1:]
            for key, fn in sections:
                # no clock sampler runs beside the serving loads: a process
                # polling NVML stalls the server's completions every ~0.5 s
                # (p99 at 0.8x load 80-130 ms with a 10 ms poller, 7-17 ms
                # without, on one GPU in one run)
                unsampled = key == "serving"
                if unsampled:
                    smi.pause()
                t_sec = time.perf_counter()
                try:
                    extras[key] = fn()
                except Exception as e:  # noqa: BLE001 -- recorded in the JSON line
                    extras[key] = {"error": f"{type(e).__name__}: {e}"}
                    torch.cuda.synchronize()
                    torch.cuda.empty_cache()
                smi.section(key, t_sec, time.perf_counter(),
                            note="sampler paused: NVML polling stalls the server" if unsampled else None)
                if unsampled:
                    smi.resume()

    # ---- roofline of the dominant kernel (the SpMV)
    alg = model.algorithmic_bytes(nrows, ncols, nnz, inf.nchunks, C, 8, 8, inf.has_perm)
    achieved = alg / kern_s / 1e9
    wl_key = f"{W['name']}:N{nrows}"
    traffic, _ = lookup_traffic(wl_key)
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic,
            "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback",
            "kernel": kernel_name(best, C, inf),
            "kernel_avg_us": round(kern_s * 1e6, 3), "algorithmic_bytes_per_launch": alg}
    nnzr = nnz / nrows
    bal = model.balance_sell(1.0 / nnzr, inf.beta, nnzr)
    extras["paper_model"] = {
        "beta": inf.beta, "nnzr": round(nnzr, 3), "zeta": round(inf.zeta, 3),
        "balance_bytes_per_flop": round(bal, 4),
        "bound_gflops_b_read": round(model.roofline(b_read, bal), 1),
        "frac_of_model_bound": round(value / n_gpus / model.roofline(b_read, bal), 4),
        "model_bytes_per_launch": int(model.paper_model_bytes(nnz, inf.beta, nrows, ncols))}
    extras["b_read_gbs"] = round(b_read, 1)
    extras["gather_peak_ggps"] = round(gather_gps, 1)
    # the FP64 pipe's rate: the FMA loop of sell_bench_fma64, or the same
    # matrix multiplying 8 vectors (one FMA per stored nonzero and vector),
    # whichever is higher -- inside the SpMMV the pipe delivers more than a
    # loop of nothing but FMAs shows
    k8 = (extras.get("spmmv_f64") or {}).get("k8", {}).get("gflops", 0.0) / 1e3
    fp64_rate = max(fma_tf, k8)
    extras["fp64_fma_peak_tflops"] = round(fma_tf, 3)
    extras["fp64_fma_bench"] = fma
    extras["fp64_rate_tflops"] = {"value": round(fp64_rate, 4), "fma_loop": round(fma_tf, 4), "spmmv_k8": round(k8, 4)}
    extras["fp64_pipe_frac"] = round(flops / kern_s / 1e12 / fp64_rate, 4)
    extras["build_ms"] = round(build_ms, 2)
    extras["tuned"] = {"C": C, "sigma": sigma, "block": best.block, "unroll": best.unroll,
                       "pipeline": best.pipeline}
    extras["sweep"] = sweep
    extras["device"] = dev_name

    cb = None
    if rank == 0 and not args.no_cpu and ws == 1:
        t_sec = time.perf_counter()
        cb = cpu_baseline(A_host, x, W["name"])
        smi.section("cpu_baseline", t_sec, time.perf_counter())
    nvml.stop()
    smi.stop()
    extras["clocks_by_section"] = smi.by_section()
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "GF/s",
            "n_gpus": n_gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(step_s * 1e3, 5), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": W["desc"], "C": C, "sigma": sigma, "nrows": nrows, "nnz": nnz,
                       "beta": round(inf.beta, 6), "stored": inf.stored,
                       "l2": f"inputs larger than L2: the matrix streams {alg / 1e9:.2f} GB per step "
                             f"(L2 {L2_BYTES / 2 ** 20:.0f} MiB), no flush needed",
                       "parallelism": f"replicas x{n_gpus}"},
            "roofline": roof, "cpu_baseline": cb, "e2e": e2e, "gpu_launches": args.steps,
            "clocks": clocks,
        }
        line.update(extras)
        line["summary"] = compact_summary(line, extras)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_sharded(args):
    """One matrix split by rows over the ranks (dist.shard_rows: whole sorting
    windows and chunks per rank).  A step is one distributed SpMV: the
    allgather of x (NCCL), then every rank's own rows; the job's rate is the
    global flops over the slowest rank's time (strong scaling)."""
    import torch
    from paper_1307_6209_gb300 import build as cuda_build
    from paper_1307_6209_gb300 import dist as sdist
    from paper_1307_6209_gb300 import model, sell, synth

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    cuda_build.build()
    sell.load()
    W = workload(args)
    C, sigma = args.C or 128, args.sigma or 1
    stream = torch.cuda.Stream()
    peak, peak_src = load_peaks()
    with torch.cuda.stream(stream):
        A = W["device"]() if W["device"] is not None else to_device(W["host"]())
        N, nnz = int(A.nrows), int(A.rpt[-1])
        bounds = sdist.shard_rows(N, sigma, C, ws, rpt=A.rpt.cpu().numpy())
        shard = sdist.build_shard(A, bounds, rank, C=C, sigma=sigma, stream=stream)
        del A
        torch.cuda.empty_cache()
        sell.sell_set_launch(shard.handle, args.block or 128, args.unroll or 4,
                             args.pipeline if args.pipeline is not None else 1)
        r0, r1 = shard.rows
        x = torch.from_numpy(synth.vector(N, seed=0)).cuda()
        x_local = x[r0:r1].contiguous()
        del x
        y_local = torch.empty(r1 - r0, dtype=torch.float64, device="cuda")
        gather = (lambda xl: xl) if ws == 1 else None

        def step():
            sdist.sharded_spmv(shard, x_local, y_local, gather=gather, stream=stream)
        for _ in range(args.warmup):
            step()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t_start.record(stream)
        for a, b in ev:
            a.record(stream)
            step()
            b.record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    total_s = t_start.elapsed_time(t_end) * 1e-3
    step_s = sdist.max_over_ranks(total_s, device="cuda") / args.steps
    loc_s = sum(a.elapsed_time(b) for a, b in ev) * 1e-3 / args.steps
    inf = shard.handle.info
    alg = model.algorithmic_bytes(inf.nrows, inf.ncols, inf.nnz, inf.nchunks, C, 8, 8, inf.has_perm)
    if rank == 0:
        value = 2.0 * nnz / step_s / 1e9
        line = {"metric": METRIC, "value": round(value, 2), "unit": "GF/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(step_s * 1e3, 5), "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": W["desc"], "C": C, "sigma": sigma, "nrows": N, "nnz": nnz,
                           "parallelism": f"rows x{ws} (allgather of x, then the local rows)",
                           "rank0_rows": [r0, r1]},
                "roofline": {"bound": "hbm", "achieved": round(alg / loc_s / 1e9, 1), "peak": peak, "unit": "GB/s",
                             "frac": round(alg / loc_s / 1e9 / peak, 4), "traffic": None,
                             "peak_source": peak_src,
                             "note": "rank 0's step (allgather + local SpMV) against its local algorithmic bytes"},
                "cpu_baseline": None, "e2e": None, "gpu_launches": args.steps}
        print(json.dumps(line), flush=True)
    shard.handle.free()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.section:
        return run_section(args)
    if args.shard == "rows":
        return run_sharded(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
