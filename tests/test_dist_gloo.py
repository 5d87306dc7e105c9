"""The multi-process paths on CPU ranks (gloo, world size 2).

* Weak scaling (what bench.py does under torchrun): the job throughput is the
  sum of the ranks' work over the slowest rank's time.
* Row sharding of one matrix: the ranks' formats are exactly the pieces of
  the global format (no sorting window or chunk crosses a boundary), and
  dist.sharded_spmv -- one allgather of x over gloo, then the rank's own rows,
  here with the oracle's Listing "sell" as the local product -- gives the
  global product bit for bit.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, results):
    import torch.distributed as dist

    import oracle
    from paper_1307_6209_gb300 import dist as sdist
    from paper_1307_6209_gb300 import synth

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = {}
        # weak scaling: units (100, 200) over max time (1.5 s)
        out["tp"] = sdist.weak_scaling_throughput(100.0 * (rank + 1), 0.5 + rank)

        # row sharding of one matrix
        A = synth.lognormal(5003, seed=4, cap=400)
        x = synth.vector(A.ncols, seed=5)
        C, sigma = 32, 256
        bounds = sdist.shard_rows(A.nrows, sigma, C, world, rpt=A.rpt)
        r0, r1 = bounds[rank]
        S = sdist.slice_rows(A, r0, r1)
        Fs = oracle.sell_build(S, C, sigma)
        F = oracle.sell_build(A, C, sigma)
        c0, c1 = r0 // C, r0 // C + Fs["nchunks"]
        out["pieces"] = bool(
            np.array_equal(Fs["cs"], F["cs"][c0:c1 + 1] - F["cs"][c0])
            and Fs["val"].tobytes() == F["val"][F["cs"][c0]:F["cs"][c1]].tobytes()
            and np.array_equal(Fs["col"], F["col"][F["cs"][c0]:F["cs"][c1]])
            and np.array_equal(Fs["perm"] + r0, F["perm"][r0:r1]))

        # the package's sharded product: each rank owns the slice of x
        # matching its rows; one allgather, then the local rows
        mine = torch.from_numpy(x[r0:r1].copy())
        shard = sdist.RowShard(bounds, rank)
        seen = {}

        def local_product(xg, _y):
            seen["x"] = xg.numpy().tobytes() == x.tobytes()
            return torch.from_numpy(oracle.sell_spmv(Fs, xg.numpy()))
        y_local = sdist.sharded_spmv(shard, mine, product=local_product).numpy()
        out["x_gathered"] = seen["x"]
        width = max(b - a for a, b in bounds)
        ypad = torch.zeros(width, dtype=torch.float64)
        ypad[:y_local.shape[0]] = torch.from_numpy(y_local)
        yparts = [torch.empty(width, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(yparts, ypad)
        y = torch.cat([p[:b - a] for p, (a, b) in zip(yparts, bounds)]).numpy()
        out["y_equal"] = y.tobytes() == oracle.csr_spmv(A, x).tobytes()
        out["bounds"] = bounds
        results[rank] = out
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_gloo(world):
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as m:
        results = m.dict()
        mp.spawn(_worker, args=(world, port, results), nprocs=world, join=True)
        res = dict(results)
    for r in range(world):
        # units 100, 200, ... over the slowest rank's 0.5 + (world - 1) seconds
        assert res[r]["tp"] == pytest.approx(100.0 * world * (world + 1) / 2 / (0.5 + world - 1))
        assert res[r]["pieces"], f"rank {r}: shard format is not a piece of the global format"
        assert res[r]["x_gathered"], f"rank {r}: the allgather did not rebuild x"
        assert res[r]["y_equal"], f"rank {r}: sharded product differs"
    b = res[0]["bounds"]
    assert b[0][0] == 0 and b[-1][1] == 5003 and all(x % 256 == 0 for x, _ in b)


def test_shard_rows_alignment():
    from paper_1307_6209_gb300 import dist as sdist
    for n, sigma, C, w in [(10000, 256, 32, 3), (1000, 1, 32, 4), (777, 10 ** 9, 64, 2), (0, 1, 32, 2)]:
        b = sdist.shard_rows(n, sigma, C, w)
        assert b[0][0] == 0 and b[-1][1] == n and len(b) == w
        step = np.lcm(max(1, min(sigma, n) if n else 1), C)
        assert all(a <= c for (a, c) in b)
        assert all(a % step == 0 or a == n for a, _ in b)


def test_shard_rows_balances_nonzeros():
    """With the row offsets given, every shard holds its share of the nonzeros
    to within one block of whole windows and chunks."""
    from paper_1307_6209_gb300 import dist as sdist
    from paper_1307_6209_gb300 import synth
    A = synth.lognormal(20000, seed=6, cap=1000)
    for sigma, C, w in [(256, 32, 4), (1, 32, 5), (4096, 64, 3)]:
        b = sdist.shard_rows(A.nrows, sigma, C, w, rpt=A.rpt)
        step = int(np.lcm(min(sigma, A.nrows), C))
        blk = max(int(A.rpt[min(i + step, A.nrows)] - A.rpt[i]) for i in range(0, A.nrows, step))
        for k, (r0, r1) in enumerate(b):
            assert r0 % step == 0 and (r1 % step == 0 or r1 == A.nrows)
            assert abs(int(A.rpt[r1]) - A.nnz * (k + 1) / w) <= blk
