"""The autotuner and the profiling tool: the tuner measures every candidate,
returns one of them, caches it by matrix signature, and the tuned handle
gives the same bits as any other format (the choice is a speed choice only)."""
import json

import pytest

from paper_1307_6209_gb300 import synth

pytestmark = pytest.mark.gpu


def test_tune_candidates_cache_and_invariance(tmp_path):
    import torch
    from paper_1307_6209_gb300 import autotune, sell

    A = synth.lognormal(20000, seed=11, cap=600)
    cache = str(tmp_path / "tune.json")
    kw = dict(Cs=(32, 64), sigmas=(1, 4096), blocks=(128, 256), unrolls=(1, 4), pipelines=(0, 1, 2), keep=2,
              reps=3, cache=cache)
    r = autotune.tune(A, **kw)
    assert not r.cached
    assert {(f["C"], f["sigma"]) for f in r.formats} == {(32, 1), (32, 4096), (64, 1), (64, 4096)}
    best = r.best
    assert (best.C, best.sigma) in {(f["C"], f["sigma"]) for f in r.formats}
    assert best.block in (128, 256) and best.unroll in (1, 4) and best.pipeline in (0, 1, 2)
    assert min(l["us"] for l in r.launches) == pytest.approx(best.us)
    # the second call is answered from the cache
    r2 = autotune.tune(A, **kw)
    assert r2.cached and (r2.best.C, r2.best.sigma, r2.best.block) == (best.C, best.sigma, best.block)
    assert json.load(open(cache))
    # the tuned handle computes the same bits as a plain SELL-32-1 handle
    h = autotune.build_tuned(A, best)
    h0 = sell.sell_build(A, C=32, sigma=1)
    x = torch.from_numpy(synth.vector(A.ncols, seed=1)).cuda()
    y, y0 = (torch.empty(A.nrows, dtype=torch.float64, device="cuda") for _ in range(2))
    sell.sell_spmv(h, x, y)
    sell.sell_spmv(h0, x, y0)
    torch.cuda.synchronize()
    assert y.cpu().numpy().tobytes() == y0.cpu().numpy().tobytes()


def test_tune_batch_picks_a_candidate():
    from paper_1307_6209_gb300 import autotune
    samples = [synth.banded(3000 + 500 * i, seed=i) for i in range(4)] + \
              [synth.lognormal(4000 + 300 * i, seed=10 + i, cap=300) for i in range(4)]
    best, table = autotune.tune_batch(samples, Cs=(32, 64), sigmas=(1, 256), reps=3)
    assert len(table) == 4 and all(t["us"] > 0 for t in table)
    assert best["us"] == min(t["us"] for t in table)


def test_profile_case_runs(capsys):
    from paper_1307_6209_gb300 import profile_case
    assert profile_case.main(["--matrix", "stencil27", "--n", "24", "--store", "bf16", "--pipeline", "1",
                              "--unroll", "8", "--reps", "2"]) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["nnz"] == (3 * 24 - 2) ** 3 and line["us"] > 0 and line["store"] == "bf16"


def test_profile_case_batch_runs(capsys):
    from paper_1307_6209_gb300 import profile_case
    assert profile_case.main(["--batch", "4", "--store", "f32", "--C", "32", "--sigma", "256", "--k", "4",
                              "--reps", "2"]) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["batch"] == 4 and line["k"] == 4 and line["us"] > 0
    assert 0 < line["beta"] <= 1 and line["nnz"] <= line["stored"]


def test_tune_plan_measures_every_launch_and_keeps_the_bits():
    """tune_plan times every (block size, right-hand-side width) of a batch
    plan and returns one of them; the plan run with the choice gives the
    same bits as the default plan."""
    import torch
    from paper_1307_6209_gb300 import autotune, sell

    hs = [sell.sell_build(synth.banded(3000 + 500 * i, seed=i), C=32, sigma=256, store_type=sell.SELL_F32)
          for i in range(6)]
    k = 8
    items = [(h, torch.rand((h.info.ncols, k), dtype=torch.float32, device="cuda"),
              torch.empty((h.info.nrows, k), dtype=torch.float32, device="cuda"), 0) for h in hs]
    best, table = autotune.tune_plan(items, k, reps=2)
    assert {(c["tile"], c["rhs"]) for c in table} == {(t, w) for t in (64, 128, 256) for w in (8, 4)}
    assert best["us"] == min(c["us"] for c in table)
    plan = sell.sell_batch_create(items)
    plan.run()
    torch.cuda.synchronize()
    ref = [Y.clone() for _, _, Y, _ in items]
    flag = {8: 0, 4: sell.SELL_SPMV_RHS_BLOCK4}[best["rhs"]]
    tuned = sell.sell_batch_create([(h, X, Y, flag) for h, X, Y, _ in items])
    tuned.set_launch(best["tile"])
    for _, _, Y, _ in items:
        Y.fill_(float("nan"))
    tuned.run()
    torch.cuda.synchronize()
    assert all(torch.equal(Y, r) for (_, _, Y, _), r in zip(items, ref))
