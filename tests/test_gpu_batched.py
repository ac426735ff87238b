"""The batched persistent launch (many densities, one launch per path family)
through the C ABI: each instance matches the oracle, matches the same
instance run alone bit for bit when the tiling is the same, and the call can
be captured in a CUDA graph and replayed."""
import numpy as np
import pytest

import oracle
import workloads
from kde_testutil import TOL_FP32, TOL_SPLIT, rel_linf, sample_cells

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2004_13653_gb300 as kde  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kde.load(build_if_stale=True)


def _mixed(seed=600, count=12):
    rng = np.random.default_rng(seed)
    kernels = [oracle.GAUSSIAN, oracle.EPANECHNIKOV, oracle.QUARTIC, oracle.GAUSSIAN,
               oracle.TRICUBE, oracle.GAUSSIAN]
    wls = []
    for k in range(count):
        n = [0, 1, 777, 3000, 5001, 12000][k % 6]
        nx, ny = int(rng.integers(20, 300)), int(rng.integers(20, 300))
        cell = float(rng.uniform(5, 20))
        h = float(rng.uniform(2, 8)) * cell
        wl = workloads.random_points(seed + k, max(n, 1), min(nx, ny) * cell, cell, nx, ny, h,
                                     kernels[k % len(kernels)])
        if n == 0:
            wl.local = wl.local[:0]
            wl.w = wl.w[:0]
        wls.append(wl)
    return wls


def _dev(wl):
    return dict(points=torch.as_tensor(np.ascontiguousarray(wl.xy).reshape(-1, 2),
                                       dtype=torch.float64, device="cuda"),
                weights=torch.as_tensor(wl.w, dtype=torch.float32, device="cuda"),
                origin=wl.origin, cell=wl.cell, nx=wl.nx, ny=wl.ny, h=wl.h, kernel=wl.kernel)


def _tol(wl):
    return TOL_SPLIT if wl.kernel == oracle.GAUSSIAN else TOL_FP32


def test_mixed_batch_matches_oracle_and_single_calls():
    wls = _mixed()
    insts = [_dev(wl) for wl in wls]
    outs = kde.grid_batched(insts, flags=kde.FLAG_SYNC, split_k=2, tile_n=256)
    for wl, d, F in zip(wls, insts, outs):
        F = F.cpu().numpy()
        ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, wl.kernel)
        if wl.n == 0 or not ref.any():
            assert not F.any()
        else:
            assert rel_linf(F, ref) <= _tol(wl), (wl.name, wl.kernel)
        alone = kde.grid(d["points"], d["weights"], wl.origin, wl.cell, wl.nx, wl.ny, wl.h,
                         wl.kernel, flags=kde.FLAG_SYNC, split_k=2, tile_n=256).cpu().numpy()
        assert np.array_equal(F, alone), (wl.name, wl.kernel)


def test_graph_capture_and_replay():
    wls = _mixed(seed=650, count=8)
    insts = [_dev(wl) for wl in wls]
    outs = [torch.full((wl.ny, wl.nx), -1.0, device="cuda") for wl in wls]
    for d, o in zip(insts, outs):
        d["out"] = o
    kde.grid_batched(insts, flags=kde.FLAG_SYNC)          # grows the workspace
    eager = [o.clone() for o in outs]
    for o in outs:
        o.fill_(-1.0)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            kde.grid_batched(insts, stream=s)
    torch.cuda.synchronize()
    for o in outs:
        o.fill_(-1.0)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    for a, b in zip(eager, outs):
        assert torch.equal(a, b)


def test_more_instances_than_one_launch_holds():
    rng = np.random.default_rng(700)
    wls = [workloads.random_points(700 + k, int(rng.integers(1, 200)), 500.0, 10.0, 50, 50, 30.0,
                                   oracle.GAUSSIAN if k % 2 else oracle.EPANECHNIKOV)
           for k in range(300)]
    outs = kde.grid_batched([_dev(wl) for wl in wls], flags=kde.FLAG_SYNC)
    for k in (0, 1, 255, 256, 299):
        wl = wls[k]
        ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, wl.kernel)
        if not ref.any():
            assert not outs[k].cpu().numpy().any()
        else:
            assert rel_linf(outs[k].cpu().numpy(), ref) <= _tol(wl)


def test_config4_batch_sampled():
    """256 instances: point counts log-uniform 1e4..2e6, grids 128^2..2048^2,
    h 50..800 m, Gaussian / Epanechnikov; sampled cells of every 16th
    instance against the oracle."""
    wls = workloads.config4_instances()
    insts = [_dev(wl) for wl in wls]
    outs = kde.grid_batched(insts, flags=kde.FLAG_SYNC)
    for k in range(0, 256, 16):
        wl = wls[k]
        F = outs[k].cpu().numpy()
        cells = sample_cells(F, 48, seed=k, neighbourhood=4)
        ref = oracle.kde_cells(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, wl.kernel,
                               cells)
        assert rel_linf(F.reshape(-1)[cells], ref) <= _tol(wl), (k, wl.kernel, wl.n)


_TILINGS = [dict(flags=kde.FLAG_CTA_PAIR, tile_n=256, stage_points=64, k_chunk=256, split_k=2),
            dict(flags=kde.FLAG_ONE_CTA, tile_n=128, stage_points=64, k_chunk=256, split_k=3),
            dict(flags=kde.FLAG_ONE_CTA, tile_n=256, stage_points=32, k_chunk=128, split_k=1),
            dict(flags=kde.FLAG_ONE_CTA, tile_n=128, stage_points=32, k_chunk=96, split_k=2)]


def test_tiled_batch_families_match_oracle_and_single_calls():
    """Per-instance tilings (kde_grid_batched_tiled): the Gaussian instances
    fall into four tile families, one launch each; every instance matches the
    oracle and, bit for bit, the same instance run alone with its tiling."""
    wls = _mixed(seed=660, count=12)
    insts = [_dev(wl) for wl in wls]
    tilings = [_TILINGS[k % 4] if wl.kernel == oracle.GAUSSIAN else None
               for k, wl in enumerate(wls)]
    outs = kde.grid_batched(insts, flags=kde.FLAG_SYNC, tilings=tilings)
    for wl, d, F, tl in zip(wls, insts, outs, tilings):
        F = F.cpu().numpy()
        ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, wl.kernel)
        if wl.n == 0 or not ref.any():
            assert not F.any()
            continue
        assert rel_linf(F, ref) <= _tol(wl), (wl.name, wl.kernel, tl)
        if tl is not None:
            alone = kde.grid(d["points"], d["weights"], wl.origin, wl.cell, wl.nx, wl.ny, wl.h,
                             wl.kernel, path="tc_split16", flags=kde.FLAG_SYNC | tl["flags"],
                             tile_n=tl["tile_n"], stage_points=tl["stage_points"],
                             k_chunk=tl["k_chunk"], split_k=tl["split_k"]).cpu().numpy()
            assert np.array_equal(F, alone), (wl.name, tl)


def test_autotuned_batch_replays_in_a_graph(tmp_path):
    """The autotuner's per-class tilings feed the batch; the tiled call is
    captured in a CUDA graph and its replay matches the eager call and the
    oracle."""
    from paper_2004_13653_gb300 import autotune
    wls = _mixed(seed=670, count=8)
    insts = [_dev(wl) for wl in wls]
    tilings = autotune.tune_batch(insts, cache_path=str(tmp_path / "tune.json"))
    assert all((t is None) == (wl.kernel != oracle.GAUSSIAN) for t, wl in zip(tilings, wls))
    outs = [torch.full((wl.ny, wl.nx), -1.0, device="cuda") for wl in wls]
    for d, o in zip(insts, outs):
        d["out"] = o
    kde.grid_batched(insts, flags=kde.FLAG_SYNC, tilings=tilings)
    eager = [o.clone() for o in outs]
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            kde.grid_batched(insts, stream=s, tilings=tilings)
    torch.cuda.synchronize()
    for o in outs:
        o.fill_(-1.0)
    g.replay()
    torch.cuda.synchronize()
    for wl, a, b in zip(wls, eager, outs):
        assert torch.equal(a, b)
        ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, wl.kernel)
        if ref.any():
            assert rel_linf(b.cpu().numpy(), ref) <= _tol(wl)
