"""The reference arm of bench.py (the FP64 oracle on the host cores) keeps the
JSON-line contract on a small workload, on the CPU: one line with the metric,
unit, config and a cpu_baseline describing the run, e2e with no copies, and
nothing from ranks other than 0."""
import argparse
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import bench
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--points", "20",
        "--grid", "256", "--steps", "2", "--warmup", "1"]


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    r = subprocess.run(ARGS, capture_output=True, text=True, env=env, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.strip()]


def test_reference_line_contract():
    lines = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["dtype"] == "f64" and d["data"] == "synthetic" and d["vs_baseline"] is None
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["unit"] == d["unit"] and cb["sample"]
    # the extrapolation is the sampled rate applied to the whole grid
    n, cells = 20 * 500, 256 * 256
    assert cb["extrapolated_full_grid_s"] == pytest.approx(n * cells / (d["value"] * 1e9),
                                                           rel=1e-9)
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_other_ranks_print_nothing():
    assert _run({"RANK": "1", "WORLD_SIZE": "2"}) == []


def test_cpu_baseline_leg_runs_on_the_host():
    """The oracle leg of the default run (rank 0, N = 1) on a 2000-point, 64^2
    case, given the oracle's own grid rounded to FP32 in place of the GPU's."""
    torch = pytest.importorskip("torch")
    args = argparse.Namespace(points=4, grid=64, h_m=0.0, cpu_cells=100)
    wl, ll, corner, lat0 = bench.make_workload(args)
    xy = oracle.mercator(ll, lat0)
    origin = oracle.mercator([corner], lat0)[0]
    F = oracle.kde_grid(xy, wl.w, origin, wl.cell, wl.nx, wl.ny, wl.h, oracle.GAUSSIAN)
    out = torch.as_tensor(np.asarray(F, np.float32))
    cb, (cells, ref) = bench.cpu_baseline(args, wl, origin, ll, lat0, out)
    assert len(cells) == 100 and cb["kind"] == "oracle" and cb["cores"] >= 1
    assert cb["unit"] == bench.UNIT and cb["value"] > 0
    assert cb["gpu_err_rel_linf_on_sample"] < 1e-6
    assert cb["extrapolated_full_grid_s"] == pytest.approx(
        wl.n * wl.nx * wl.ny / (cb["value"] * 1e9), rel=1e-9)
