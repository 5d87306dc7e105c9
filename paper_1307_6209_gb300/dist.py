"""Multi-process helpers (one process per GPU).

Two ways the SpMV spreads over several GPUs:

* Independent problems (the benchmark's weak scaling): every rank multiplies
  its own matrix; the only collective is the timing reduction (maximum of the
  ranks' elapsed times), and the job's throughput is the sum of the ranks'
  work divided by that maximum.
* One matrix split by rows (`shard_rows`, `build_shard`, `sharded_spmv`):
  every rank owns a contiguous block of whole sorting windows (so no window,
  and no chunk, crosses a rank boundary and the ranks' formats are exactly the
  pieces of the global format), a slice of x and the matching slice of y.
  The one exchange per product is an allgather of x; each rank then computes
  its own rows with no reduction.  (The paper leaves distributed-memory SpMV
  to future work, Sec. 6.)
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass


def env():
    """(world_size, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_throughput(units_per_rank: float, seconds: float, device=None) -> float:
    """Job throughput: the units of every rank over the slowest rank's time."""
    import torch
    import torch.distributed as dist
    tmax = max_over_ranks(seconds, device)
    if not dist.is_initialized():
        return units_per_rank / tmax
    t = torch.tensor([float(units_per_rank)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item()) / tmax


def shard_rows(nrows: int, sigma: int, C: int, world: int, rpt=None):
    """Split rows [0, nrows) into `world` contiguous ranges whose boundaries are
    multiples of lcm(min(sigma, nrows), C) -- whole sorting windows and whole
    chunks -- balanced by nonzeros when `rpt` (CRS row offsets) is given."""
    w = max(1, min(sigma, nrows) if nrows else 1)
    step = w * C // math.gcd(w, C)
    nblk = (nrows + step - 1) // step
    if rpt is not None and nrows > 0:
        total = int(rpt[nrows])
        bounds = [0]
        for k in range(1, world):
            target = total * k / world
            # first block boundary whose prefix reaches the target
            lo, hi = bounds[-1] // step, nblk
            while lo < hi:
                mid = (lo + hi) // 2
                if int(rpt[min(mid * step, nrows)]) < target:
                    lo = mid + 1
                else:
                    hi = mid
            bounds.append(min(max(lo * step, bounds[-1]), nrows))
        bounds.append(nrows)
    else:
        per = (nblk + world - 1) // world
        bounds = [min(k * per * step, nrows) for k in range(world)] + [nrows]
    return [(bounds[k], bounds[k + 1]) for k in range(world)]


def slice_rows(A, r0: int, r1: int):
    """Rows [r0, r1) of a CSR matrix (numpy or torch arrays) as a CSR matrix
    with all the columns: the local matrix of the rank that owns those rows."""
    a, b = int(A.rpt[r0]), int(A.rpt[r1])
    return type(A)(r1 - r0, A.ncols, A.rpt[r0:r1 + 1] - A.rpt[r0], A.col[a:b], A.val[a:b])


@dataclass
class RowShard:
    """One rank's part of a row-sharded square matrix: the row ranges of all
    ranks (`bounds`, from shard_rows), this rank's index, and the SELL-C-sigma
    handle of its rows (built with the global C and sigma, so that it is the
    matching piece of the global format)."""
    bounds: list
    rank: int
    handle: object = None

    @property
    def rows(self):
        return self.bounds[self.rank]


def build_shard(A, bounds, rank: int, C: int = 32, sigma: int = 1, store_type: int = 0, stream=None) -> RowShard:
    """Build this rank's handle from the global CSR (numpy or CUDA arrays)."""
    from . import sell
    r0, r1 = bounds[rank]
    h = sell.sell_build(slice_rows(A, r0, r1), C=C, sigma=sigma, store_type=store_type, stream=stream)
    return RowShard(list(bounds), rank, h)


def allgather_x(x_local, bounds, group=None):
    """The full x from every rank's slice: one all_gather of the slices, each
    padded to the longest one (NCCL for CUDA tensors, gloo for CPU ones);
    rank k's slice is x[bounds[k][0]:bounds[k][1]]."""
    import torch
    import torch.distributed as dist
    width = max(b - a for a, b in bounds)
    pad = torch.zeros(width, dtype=x_local.dtype, device=x_local.device)
    pad[:x_local.shape[0]] = x_local
    parts = [torch.empty_like(pad) for _ in bounds]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:b - a] for p, (a, b) in zip(parts, bounds)])


def sharded_spmv(shard: RowShard, x_local, y_local=None, group=None, gather=None, product=None, stream=None):
    """y_local = A[rows of this rank, :] x for a square matrix whose rows and
    x are split by `shard.bounds`: one exchange (the allgather of x), then the
    rank's own rows with no reduction.  The seams for testing and other
    transports: `gather(x_local) -> x` replaces the all_gather, and
    `product(x, y_local) -> y_local` the local sell_spmv (for example the
    oracle on the local CSR on CPU ranks).  Returns y_local."""
    x = gather(x_local) if gather is not None else allgather_x(x_local, shard.bounds, group)
    if product is None:
        import torch
        from . import sell
        if y_local is None:
            r0, r1 = shard.rows
            y_local = torch.empty(r1 - r0, dtype=x.dtype, device=x.device)
        sell.sell_spmv(shard.handle, x, y_local, stream=stream)
        return y_local
    return product(x, y_local)
