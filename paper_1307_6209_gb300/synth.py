"""Seeded synthetic sparse matrices and vectors (CSR, numpy).

This module only generates inputs.  It holds none of the SELL-C-sigma
arithmetic, so both the CUDA library's tests and the CPU oracle can be fed from
it without sharing any of the method's code.

The matrices stand in for the University of Florida collection used by the
paper (Sec. 2.2, Table "table:matrices"), which is not available here:

* ``laplace2d``   5-point Laplacian on an nx x ny grid (diagonal 4, neighbours -1).
* ``stencil27``   27-point stencil on an n^3 grid (diagonal 26, neighbours -1,
                  optionally perturbed by a seeded factor 1 + p*U(-1,1) so that
                  rounding to binary32/bfloat16 is not exact).
* ``lognormal``   random square matrix; row lengths lognormal with the given mean
                  and log-standard deviation, rounded to nearest and clamped to
                  [1, cap]; distinct uniform columns per row, sorted; values N(0,1).
* ``banded``      random banded matrix: each row has U{lo..hi} distinct columns
                  within +-bandwidth of the diagonal; values N(0,1).
* ``beta_worst``  the worst case of Sec. 3.4 (Eq. "betaworst"): one full row and
                  C-1 single-entry rows in every chunk of C rows.
* ``random_csr``  small random matrix with a given density (empty rows allowed).
* ``dense``       a dense n x m matrix stored as CSR.
* ``long_row``    short rows plus one very long row (a webbase-1M-like profile).

All randomness comes from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    nrows: int
    ncols: int
    rpt: np.ndarray  # int64[nrows + 1]
    col: np.ndarray  # int32[nnz], ascending inside each row
    val: np.ndarray  # float64[nnz]

    @property
    def nnz(self) -> int:
        return int(self.rpt[-1]) if self.nrows > 0 else 0

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.rpt)

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.nrows, self.ncols), np.float64)
        rows = np.repeat(np.arange(self.nrows), self.row_lengths())
        d[rows, self.col.astype(np.int64)] = self.val
        return d


def _from_lengths(rl: np.ndarray, ncols: int, col: np.ndarray, val: np.ndarray) -> CSR:
    rpt = np.zeros(rl.shape[0] + 1, np.int64)
    np.cumsum(rl, out=rpt[1:])
    return CSR(int(rl.shape[0]), int(ncols), rpt, np.ascontiguousarray(col, np.int32),
               np.ascontiguousarray(val, np.float64))


def laplace2d(nx: int, ny: int | None = None) -> CSR:
    ny = nx if ny is None else ny
    n = nx * ny
    idx = np.arange(n, dtype=np.int64)
    gx, gy = idx % nx, idx // nx
    # neighbours in ascending column order: (y-1), (x-1), self, (x+1), (y+1)
    offs = [(-nx, gy > 0, -1.0), (-1, gx > 0, -1.0), (0, np.ones(n, bool), 4.0),
            (1, gx < nx - 1, -1.0), (nx, gy < ny - 1, -1.0)]
    cols = np.stack([idx + o for o, _, _ in offs], axis=1)
    mask = np.stack([m for _, m, _ in offs], axis=1)
    vals = np.broadcast_to(np.array([v for _, _, v in offs]), cols.shape)
    return _from_lengths(mask.sum(1), n, cols[mask], vals[mask])


def stencil27(n: int, perturb: float = 0.0, seed: int = 0, rows: int | None = None) -> CSR:
    """The 27-point stencil on an n^3 grid; with ``rows``, only its first
    ``rows`` rows (a rows x n^3 matrix whose arrays equal the prefix of the
    full matrix's, values included)."""
    N = n ** 3
    R = N if rows is None else max(0, min(int(rows), N))
    idx = np.arange(R, dtype=np.int64)
    gx, gy, gz = idx % n, (idx // n) % n, idx // (n * n)
    cols = np.empty((R, 27), np.int32)
    mask = np.empty((R, 27), bool)
    vals = np.empty((R, 27), np.float64)
    t = 0
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                ok = ((gx + dx >= 0) & (gx + dx < n) & (gy + dy >= 0) & (gy + dy < n)
                      & (gz + dz >= 0) & (gz + dz < n))
                cols[:, t] = idx + dz * n * n + dy * n + dx
                mask[:, t] = ok
                vals[:, t] = 26.0 if (dx, dy, dz) == (0, 0, 0) else -1.0
                t += 1
    rl = mask.sum(1)
    col = cols[mask]
    del cols
    val = vals[mask]
    del vals, mask
    if perturb:
        rng = np.random.default_rng(seed)  # sequential draws: a prefix of rows gets the prefix of the values
        val *= 1.0 + perturb * rng.uniform(-1.0, 1.0, val.shape[0])
    return _from_lengths(rl, N, col, val)


def lognormal_lengths(N: int, mean: float = 16.0, sigma_ln: float = 1.2, cap: int = 2000,
                      rng=None) -> np.ndarray:
    """Row lengths whose underlying normal has mu = ln(mean) - sigma_ln^2/2, so
    that the unclamped mean is ``mean``; rounded to nearest, clamped to [1, cap]."""
    rng = np.random.default_rng(0) if rng is None else rng
    mu = np.log(mean) - 0.5 * sigma_ln * sigma_ln
    rl = np.rint(np.exp(mu + sigma_ln * rng.standard_normal(N)))
    return np.clip(rl, 1, cap).astype(np.int64)


def _distinct_sorted_columns(rl: np.ndarray, lo: np.ndarray, hi: np.ndarray, rng) -> np.ndarray:
    """For every row i draw rl[i] distinct integers uniformly from [lo[i], hi[i]),
    sorted ascending; rows are concatenated in row order.  Rows that need more
    than a quarter of their span are drawn without replacement one by one;
    the others by drawing with replacement and redrawing duplicates."""
    N = rl.shape[0]
    out = np.empty(int(rl.sum()), np.int64)
    start = np.zeros(N + 1, np.int64)
    np.cumsum(rl, out=start[1:])
    full = rl > np.maximum(hi - lo, 1) // 4
    for i in np.nonzero(full)[0]:
        out[start[i]:start[i + 1]] = lo[i] + np.sort(rng.choice(int(hi[i] - lo[i]), size=int(rl[i]),
                                                                replace=False))
    sparse_rows = np.nonzero(~full)[0]
    if sparse_rows.size:
        rls = rl[sparse_rows]
        rows = np.repeat(np.arange(sparse_rows.size, dtype=np.int64), rls)
        span = (hi - lo)[sparse_rows][rows]
        base = lo[sparse_rows][rows]
        width = int(max(1, (hi - lo)[sparse_rows].max(initial=1)))
        cols = base + rng.integers(0, np.iinfo(np.int64).max, rows.shape[0]) % span
        while True:
            key = rows * width + (cols - base)
            order = np.argsort(key, kind="stable")
            ks = key[order]
            dup = np.nonzero(ks[1:] == ks[:-1])[0] + 1
            if dup.size == 0:
                cols = cols[order]
                break
            at = order[dup]
            cols[at] = base[at] + rng.integers(0, np.iinfo(np.int64).max, at.shape[0]) % span[at]
        pos = np.repeat(start[sparse_rows], rls) + (np.arange(rows.shape[0]) - np.repeat(
            np.concatenate([[0], np.cumsum(rls)[:-1]]), rls))
        out[pos] = cols
    return out


def lognormal(N: int, mean: float = 16.0, sigma_ln: float = 1.2, cap: int = 2000,
              seed: int = 0) -> CSR:
    rng = np.random.default_rng(seed)
    cap = min(cap, N)
    rl = lognormal_lengths(N, mean, sigma_ln, cap, rng)
    col = _distinct_sorted_columns(rl, np.zeros(N, np.int64), np.full(N, N, np.int64), rng)
    val = rng.standard_normal(col.shape[0])
    return _from_lengths(rl, N, col, val)


def banded(N: int, bandwidth: int = 64, lo: int = 7, hi: int = 30, seed: int = 0) -> CSR:
    rng = np.random.default_rng(seed)
    i = np.arange(N, dtype=np.int64)
    a = np.maximum(i - bandwidth, 0)
    b = np.minimum(i + bandwidth + 1, N)
    rl = np.minimum(rng.integers(lo, hi + 1, N), b - a)
    col = _distinct_sorted_columns(rl, a, b, rng)
    val = rng.standard_normal(col.shape[0])
    return _from_lengths(rl, N, col, val)


def beta_worst(N: int, C: int, seed: int = 0) -> CSR:
    """Sec. 3.4 worst case: in every chunk of C rows the first row is full
    (N entries) and the other C-1 rows hold one entry (on the diagonal)."""
    assert N % C == 0
    rng = np.random.default_rng(seed)
    rl = np.ones(N, np.int64)
    rl[::C] = N
    cols = []
    for i in range(N):
        cols.append(np.arange(N) if i % C == 0 else np.array([i]))
    col = np.concatenate(cols)
    val = rng.uniform(-1.0, 1.0, col.shape[0])
    return _from_lengths(rl, N, col, val)


def random_csr(N: int, M: int | None = None, density: float = 0.1, seed: int = 0,
               empty_rows: float = 0.0) -> CSR:
    M = N if M is None else M
    rng = np.random.default_rng(seed)
    d = rng.random((N, M)) < density
    if empty_rows > 0:
        d[rng.random(N) < empty_rows, :] = False
    rows, cols = np.nonzero(d)
    val = rng.standard_normal(rows.shape[0])
    return _from_lengths(d.sum(1), M, cols, val)


def dense(N: int, M: int | None = None, seed: int = 0) -> CSR:
    M = N if M is None else M
    rng = np.random.default_rng(seed)
    rl = np.full(N, M, np.int64)
    col = np.tile(np.arange(M, dtype=np.int32), N)
    val = rng.standard_normal(N * M)
    return _from_lengths(rl, M, col, val)


def long_row(N: int, long_len: int, short_len: int = 3, at: int = 0, seed: int = 0) -> CSR:
    rng = np.random.default_rng(seed)
    rl = np.full(N, min(short_len, N), np.int64)
    rl[at] = min(long_len, N)
    col = _distinct_sorted_columns(rl, np.zeros(N, np.int64), np.full(N, N, np.int64), rng)
    val = rng.standard_normal(col.shape[0])
    return _from_lengths(rl, N, col, val)


def from_dense(d: np.ndarray) -> CSR:
    rows, cols = np.nonzero(d)
    return _from_lengths((d != 0).sum(1), d.shape[1], cols, d[rows, cols])


def vector(n: int, seed: int = 0, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, n)


def block(n: int, k: int, seed: int = 0) -> np.ndarray:
    """Row-major n x k block of right-hand sides, U[-1, 1]."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, (n, k))


def stencil27_device(n: int, perturb: float = 0.1, seed: int = 0, device: str = "cuda") -> CSR:
    """The 27-point stencil of ``stencil27`` generated on the GPU with torch
    (same structure and base values; the perturbation factors come from
    torch's seeded device generator, so they differ from the numpy version).
    rpt/col/val are CUDA tensors."""
    import torch

    N = n ** 3
    idx = torch.arange(N, device=device, dtype=torch.int64)
    gx, gy, gz = idx % n, (idx // n) % n, idx // (n * n)

    def span(g):
        return 3 - (g == 0).to(torch.int64) - (g == n - 1).to(torch.int64)

    rl = span(gx) * span(gy) * span(gz) if n > 1 else torch.ones(N, dtype=torch.int64, device=device)
    rpt = torch.zeros(N + 1, dtype=torch.int64, device=device)
    torch.cumsum(rl, 0, out=rpt[1:])
    nnz = int(rpt[-1])
    col = torch.empty(nnz, dtype=torch.int32, device=device)
    val = torch.empty(nnz, dtype=torch.float64, device=device)
    cnt = torch.zeros(N, dtype=torch.int64, device=device)
    start = rpt[:-1]
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                ok = ((gx + dx >= 0) & (gx + dx < n) & (gy + dy >= 0) & (gy + dy < n)
                      & (gz + dz >= 0) & (gz + dz < n))
                rows = torch.nonzero(ok, as_tuple=True)[0]
                pos = start[rows] + cnt[rows]
                col[pos] = (rows + dz * n * n + dy * n + dx).to(torch.int32)
                val[pos] = 26.0 if (dx, dy, dz) == (0, 0, 0) else -1.0
                cnt += ok.to(torch.int64)
                del ok, rows, pos
    if perturb:
        g = torch.Generator(device=device)
        g.manual_seed(seed)
        val *= 1.0 + perturb * (2.0 * torch.rand(nnz, generator=g, dtype=torch.float64, device=device) - 1.0)
    return CSR(N, N, rpt, col, val)


def _distinct_sorted_columns_device(rl, lo, hi, gen):
    """Device version of _distinct_sorted_columns (torch): rl[i] distinct
    integers uniform in [lo[i], hi[i]) per row, sorted, rows concatenated.
    Rows that need more than a quarter of their span are drawn by a random
    permutation one by one; the others with replacement plus redraws."""
    import torch
    dev = rl.device
    N = rl.shape[0]
    start = torch.zeros(N + 1, dtype=torch.int64, device=dev)
    torch.cumsum(rl, 0, out=start[1:])
    out = torch.empty(int(start[-1]), dtype=torch.int64, device=dev)
    spans = torch.clamp(hi - lo, min=1)
    full = rl > spans // 4
    for i in torch.nonzero(full, as_tuple=True)[0].tolist():
        sp = int(spans[i])
        pick = torch.randperm(sp, generator=gen, device=dev)[:int(rl[i])]
        out[int(start[i]):int(start[i + 1])] = lo[i] + torch.sort(pick).values
    keep = torch.nonzero(~full, as_tuple=True)[0]
    if keep.numel():
        rls = rl[keep]
        rows = torch.repeat_interleave(torch.arange(keep.numel(), device=dev, dtype=torch.int64), rls)
        span = spans[keep][rows]
        base = lo[keep][rows]
        width = int(max(1, int(spans[keep].max())))

        def draw(m, sp):
            r = torch.randint(0, 2 ** 62, (m,), generator=gen, device=dev, dtype=torch.int64)
            return r % sp

        off = draw(rows.shape[0], span)
        while True:
            key = rows * width + off
            key, order = torch.sort(key)
            off = off[order]
            dup = torch.nonzero(key[1:] == key[:-1], as_tuple=True)[0] + 1
            if dup.numel() == 0:
                break
            off[dup] = draw(dup.numel(), span[dup])
        first = torch.zeros(keep.numel() + 1, dtype=torch.int64, device=dev)
        torch.cumsum(rls, 0, out=first[1:])
        pos = torch.repeat_interleave(start[keep], rls) + (torch.arange(rows.shape[0], device=dev)
                                                          - torch.repeat_interleave(first[:-1], rls))
        out[pos] = base + off
    return out


def lognormal_device(N: int, mean: float = 16.0, sigma_ln: float = 1.2, cap: int = 2000, seed: int = 0,
                     device: str = "cuda") -> CSR:
    """The ``lognormal`` recipe generated with torch on the device (own seeded
    stream, so the values differ from the numpy version)."""
    import math
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    mu = math.log(mean) - 0.5 * sigma_ln * sigma_ln
    z = torch.randn(N, generator=g, device=device, dtype=torch.float64)
    rl = torch.clamp(torch.round(torch.exp(mu + sigma_ln * z)), 1, min(cap, N)).to(torch.int64)
    col = _distinct_sorted_columns_device(rl, torch.zeros(N, dtype=torch.int64, device=device),
                                          torch.full((N,), N, dtype=torch.int64, device=device), g)
    val = torch.randn(col.shape[0], generator=g, device=device, dtype=torch.float64)
    rpt = torch.zeros(N + 1, dtype=torch.int64, device=device)
    torch.cumsum(rl, 0, out=rpt[1:])
    return CSR(N, N, rpt, col.to(torch.int32), val)


def banded_device(N: int, bandwidth: int = 64, lo: int = 7, hi: int = 30, seed: int = 0,
                  device: str = "cuda") -> CSR:
    """The ``banded`` recipe generated with torch on the device."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    i = torch.arange(N, device=device, dtype=torch.int64)
    a = torch.clamp(i - bandwidth, min=0)
    b = torch.clamp(i + bandwidth + 1, max=N)
    rl = torch.minimum(torch.randint(lo, hi + 1, (N,), generator=g, device=device, dtype=torch.int64), b - a)
    col = _distinct_sorted_columns_device(rl, a, b, g)
    val = torch.randn(col.shape[0], generator=g, device=device, dtype=torch.float64)
    rpt = torch.zeros(N + 1, dtype=torch.int64, device=device)
    torch.cumsum(rl, 0, out=rpt[1:])
    return CSR(N, N, rpt, col.to(torch.int32), val)


def dense_device(n: int, m: int | None = None, seed: int = 0, device: str = "cuda") -> CSR:
    """A dense n x m matrix stored as CSR on the device (values N(0,1))."""
    import torch
    m = n if m is None else m
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    rpt = torch.arange(n + 1, device=device, dtype=torch.int64) * m
    col = torch.arange(m, device=device, dtype=torch.int32).repeat(n)
    val = torch.randn(n * m, generator=g, device=device, dtype=torch.float64)
    return CSR(n, m, rpt, col, val)


def long_row_device(N: int, long_len: int, short_len: int = 3, at: int = 0, seed: int = 0,
                    device: str = "cuda") -> CSR:
    """Short rows of ``short_len`` distinct random columns plus one row of
    ``long_len`` (a webbase-1M-like profile: the paper's Sec. 5.2 cites one
    row of 1,000,005 entries against a mean of 3.11), on the device."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    rl = torch.full((N,), min(short_len, N), dtype=torch.int64, device=device)
    rl[at] = min(long_len, N)
    col = _distinct_sorted_columns_device(rl, torch.zeros(N, dtype=torch.int64, device=device),
                                          torch.full((N,), N, dtype=torch.int64, device=device), g)
    val = torch.randn(col.shape[0], generator=g, device=device, dtype=torch.float64)
    rpt = torch.zeros(N + 1, dtype=torch.int64, device=device)
    torch.cumsum(rl, 0, out=rpt[1:])
    return CSR(N, N, rpt, col.to(torch.int32), val)


def batch_set(nmat: int = 512, seed: int = 0) -> list:
    """The batched workload's matrices as (kind, nrows, seed) triples: rows
    uniform in [1000, 200000]; even positions ``banded`` (bandwidth 64, 7-30
    entries per row), odd positions ``lognormal``; matrix i uses seed i.
    Generate each with ``banded_device`` / ``lognormal_device``."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(1000, 200001, nmat)
    return [("banded" if i % 2 == 0 else "lognormal", int(n), i) for i, n in enumerate(sizes)]
