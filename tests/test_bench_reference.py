"""bench.py's reference arm on the CPU: the oracle timed on the host cores.

Rank 0 prints exactly one JSON line with the contract's keys; any other rank
of a multi-process launch exits 0 without work or output.
"""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra, *args):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                          capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)


def test_rank0_prints_one_line_with_the_contract_keys():
    # a 40^3 stencil keeps the CPU test short; the default is the 200^3 grid
    r = _run({"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"}, "--steps", "2", "--warmup", "3", "--n", "40")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3
    assert d["value"] > 0 and d["unit"] == "GF/s" and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "GF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("27-point stencil on a 40^3 grid (N=64000, nnz=1643032)")
    assert "rows 0..63999" in d["config"]["sample"]  # the whole 40^3 matrix fits the time budget


def test_default_workload_is_the_200_cubed_stencil():
    sys.path.insert(0, ROOT)
    import bench
    old = sys.argv
    try:
        sys.argv = ["bench.py"]
        args = bench.parse_args()
    finally:
        sys.argv = old
    W = bench.workload(args)
    assert W["name"] == "stencil27" and W["nrows"] == 8_000_000 and W["nnz"] == 213_847_192
    assert W["desc"].startswith("27-point stencil on a 200^3 grid")


def test_other_ranks_exit_without_work():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--steps", "2", "--warmup", "3", "--gpus", "2")
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_cpu_baseline_leg_reports_the_oracle():
    """The cpu_baseline object of our arm's line: the oracle's CRS SpMV timed
    on the host cores, with its sample and schedule stated."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1307_6209_gb300 import synth
    A = synth.lognormal(20000, seed=1)
    cb = bench.cpu_baseline(A, synth.vector(A.ncols, seed=0), "lognormal", target_s=0.2)
    assert cb["kind"] == "oracle" and cb["unit"] == "GF/s" and cb["value"] > 0 and cb["cores"] >= 1
    assert f"({A.nnz} nnz)" in cb["sample"] and "GUIDED,1" in cb["sample"]  # zeta >= 0.4 here
