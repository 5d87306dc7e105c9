"""Row sharding of one matrix, run shard after shard on one GPU.

dist.shard_rows cuts the rows at multiples of lcm(min(sigma, N), C), so no
sorting window and no chunk crosses a shard: each shard's GPU format must be
exactly the matching piece of the global format, and dist.sharded_spmv --
with the full x that one allgather gives every rank, here handed over by its
gather seam since the shards share one process -- must give y slices that
concatenate to the global y bit for bit."""
import numpy as np
import pytest

from paper_1307_6209_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [2, 3, 5])
@pytest.mark.parametrize("C,sigma", [(32, 256), (64, 1), (128, 4096)])
def test_shards_are_pieces_and_concatenate_bitwise(world, C, sigma):
    import torch
    from paper_1307_6209_gb300 import dist as sdist
    from paper_1307_6209_gb300 import sell

    A = synth.lognormal(30011, seed=7, cap=900)
    x = torch.from_numpy(synth.vector(A.ncols, seed=8)).cuda()
    hg = sell.sell_build(A, C=C, sigma=sigma)
    G = sell.sell_export(hg)
    yg = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
    sell.sell_spmv(hg, x, yg)
    parts = []
    bounds = sdist.shard_rows(A.nrows, sigma, C, world, rpt=A.rpt)
    for rank, (r0, r1) in enumerate(bounds):
        shard = sdist.build_shard(A, bounds, rank, C=C, sigma=sigma)
        hs = shard.handle
        F = sell.sell_export(hs)
        c0, c1 = r0 // C, r0 // C + hs.info.nchunks
        assert np.array_equal(F["cs"], G["cs"][c0:c1 + 1] - G["cs"][c0])
        assert F["val"].tobytes() == G["val"][G["cs"][c0]:G["cs"][c1]].tobytes()
        assert np.array_equal(F["col"], G["col"][G["cs"][c0]:G["cs"][c1]])
        if sigma > 1:
            assert np.array_equal(F["perm"] + r0, G["perm"][r0:r1])
        ys = sdist.sharded_spmv(shard, x[r0:r1], gather=lambda xl: x)
        parts.append(ys)
        hs.free()
    torch.cuda.synchronize()
    assert torch.cat(parts).cpu().numpy().tobytes() == yg.cpu().numpy().tobytes()
    hg.free()
