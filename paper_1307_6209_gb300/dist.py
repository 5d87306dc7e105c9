"""Multi-process helpers (one process per GPU).

Two ways the SpMV spreads over several GPUs:

* Independent problems (the benchmark's weak scaling): every rank multiplies
  its own matrix; the only collective is the timing reduction (maximum of the
  ranks' elapsed times), and the job's throughput is the sum of the ranks'
  work divided by that maximum.
* One matrix split by rows: every rank owns a contiguous block of whole
  sorting windows (so no window, and no chunk, crosses a rank boundary and the
  ranks' formats are exactly the pieces of the global format), a slice of x
  and the matching slice of y.  The one exchange per product is an allgather
  of x; each rank then computes its own rows with no reduction.  (The paper
  leaves distributed-memory SpMV to future work, Sec. 6.)
"""
from __future__ import annotations

import math
import os


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
