"""Parity of the tcgen05 tensor-core path (path b, Gaussian) with the FP64
oracle, through the C ABI, on the GPU: single FP16 within 2e-3 and split-FP16
within 1e-5 (relative L-inf, normalised by max F)."""
import numpy as np
import pytest

import oracle
import workloads
from kde_testutil import TOL_FP16, TOL_SPLIT, rel_linf, sample_cells

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2004_13653_gb300 as kde  # noqa: E402

TOL = {"tc_fp16": TOL_FP16, "tc_split16": TOL_SPLIT}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kde.load(build_if_stale=True)


def run_gpu(wl, path, weights=True, flags_extra=0, **kw):
    pts = torch.as_tensor(np.ascontiguousarray(wl.xy), dtype=torch.float64, device="cuda")
    w = torch.as_tensor(wl.w, dtype=torch.float32, device="cuda") if weights else None
    out = kde.grid(pts, w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, "gaussian", path=path,
                   flags=kde.FLAG_SYNC | flags_extra, **kw)
    return out.cpu().numpy()


@pytest.mark.parametrize("path", ["tc_split16", "tc_fp16"])
@pytest.mark.parametrize("tile_n", [128, 256])
def test_config1_full_grid(path, tile_n):
    wl = workloads.config1()
    F = run_gpu(wl, path, tile_n=tile_n)
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, oracle.GAUSSIAN)
    assert rel_linf(F, ref) <= TOL[path]


@pytest.mark.parametrize("path", ["tc_split16", "tc_fp16"])
@pytest.mark.parametrize("tile_n", [128, 256])
@pytest.mark.parametrize("stage_points", [32, 64])
def test_ragged_tiles_weighted(path, tile_n, stage_points):
    """3x3 tiles with ragged edges on both axes, n not a multiple of 64,
    weights U(0.5, 2), points partly outside the grid; both stage depths
    (128-byte and 64-byte swizzled operand rows)."""
    wl = workloads.random_points(400, 3001, 5000.0, 12.5, 300, 520, 40.0, oracle.GAUSSIAN)
    F = run_gpu(wl, path, tile_n=tile_n, stage_points=stage_points)
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, oracle.GAUSSIAN)
    assert rel_linf(F, ref) <= TOL[path]


def _dense_cluster():
    """10,000 of 20,000 points inside ~5 bandwidths: every MMA step of those
    points adds to the same accumulators (the hardest case for the tensor
    core's FP32 accumulation)."""
    wl = workloads.random_points(401, 20000, 3000.0, 10.0, 256, 256, 30.0, oracle.GAUSSIAN)
    wl.local[:10000] = wl.local[:10000] * 0.05 + 1500.0
    return wl


@pytest.mark.parametrize("path,k_chunk,split_k,stage_points", [
    ("tc_split16", 128, 1, 64), ("tc_split16", 256, 3, 32), ("tc_split16", 0, 0, 0),
    ("tc_split16", 384, 7, 64), ("tc_split16", 96, 2, 32),
    ("tc_fp16", 0, 0, 0), ("tc_fp16", 4096, 2, 64), ("tc_fp16", 192, 5, 32)])
def test_dense_cluster_chunk_and_split_variants(path, k_chunk, split_k, stage_points):
    wl = _dense_cluster()
    F = run_gpu(wl, path, k_chunk=k_chunk, split_k=split_k, stage_points=stage_points)
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, oracle.GAUSSIAN)
    assert rel_linf(F, ref) <= TOL[path]


def test_unit_weights_and_single_cell():
    wl = workloads.config1()
    F = run_gpu(wl, "tc_split16", weights=False)
    ref = oracle.kde_grid(wl.xy, None, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, oracle.GAUSSIAN)
    assert rel_linf(F, ref) <= TOL_SPLIT
    one = workloads.random_points(402, 5, 50.0, 10.0, 1, 1, 30.0, oracle.GAUSSIAN)
    F1 = run_gpu(one, "tc_split16")
    r1 = oracle.kde_grid(one.xy, one.w, one.origin, one.cell, 1, 1, one.h, oracle.GAUSSIAN)
    assert rel_linf(F1, r1) <= TOL_SPLIT


@pytest.mark.parametrize("path", ["tc_split16", "tc_fp16"])
def test_config2_sampled(path):
    wl = workloads.config2()
    F = run_gpu(wl, path)
    cells = sample_cells(F, 256, seed=11)
    ref = oracle.kde_cells(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, oracle.GAUSSIAN,
                           cells)
    assert rel_linf(F.reshape(-1)[cells], ref) <= TOL[path]


def test_config3_full_size_sampled():
    """The 20M-point 4096^2 workload in the launch configuration the bench
    times (AUTO = split-FP16, automatic tiling), from lon/lat through the
    GPU projection; the oracle projects on its own and evaluates sampled
    cells including the GPU argmax neighbourhood."""
    wl = workloads.config3()
    ll, corner, lat0 = wl.lonlat()
    lonlat = torch.as_tensor(ll, dtype=torch.float64, device="cuda")
    xy = kde.project_mercator(lonlat, lat0)
    origin = oracle.mercator([corner], lat0)[0]
    w = torch.as_tensor(wl.w, dtype=torch.float32, device="cuda")
    F = kde.grid(xy, w, origin, wl.cell, wl.nx, wl.ny, wl.h, "gaussian", path="tc_split16",
                 flags=kde.FLAG_SYNC).cpu().numpy()
    del xy, lonlat
    cells = sample_cells(F, 192, seed=12)
    ref = oracle.kde_cells(oracle.mercator(ll, lat0), wl.w, origin, wl.cell, wl.nx, wl.ny, wl.h,
                           oracle.GAUSSIAN, cells)
    assert rel_linf(F.reshape(-1)[cells], ref) <= TOL_SPLIT


def test_autotuned_tiling_is_valid_and_accurate(tmp_path):
    from paper_2004_13653_gb300 import autotune
    wl = workloads.config2(n_traj=400)
    pts = torch.as_tensor(wl.xy, dtype=torch.float64, device="cuda")
    w = torch.as_tensor(wl.w, dtype=torch.float32, device="cuda")
    cache = str(tmp_path / "tune.json")
    opts = autotune.tune(pts, w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, "tc_split16",
                         cache_path=cache)
    assert opts in autotune.CANDIDATES["tc_split16"]
    assert autotune.tune(pts, w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, "tc_split16",
                         cache_path=cache) == opts  # served from the cache
    tiling = dict(opts)
    flags = kde.FLAG_SYNC | tiling.pop("flags")
    F = kde.grid(pts, w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, "gaussian", path="tc_split16",
                 flags=flags, **tiling).cpu().numpy()
    cells = sample_cells(F, 128, seed=13)
    ref = oracle.kde_cells(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, oracle.GAUSSIAN,
                           cells)
    assert rel_linf(F.reshape(-1)[cells], ref) <= TOL_SPLIT


@pytest.mark.parametrize("path", ["tc_split16", "tc_fp16"])
def test_cta_pair_config1_and_ragged(path):
    """256 x 256 tiles on CTA pairs (cta_group::2): each CTA generates its own
    128 rows of A and of B; ragged tiles on both axes."""
    for wl in (workloads.config1(),
               workloads.random_points(410, 3001, 5000.0, 12.5, 300, 520, 40.0, oracle.GAUSSIAN)):
        F = run_gpu(wl, path, flags_extra=kde.FLAG_CTA_PAIR)
        ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h,
                              oracle.GAUSSIAN)
        assert rel_linf(F, ref) <= TOL[path]


@pytest.mark.parametrize("k_chunk,split_k", [(128, 1), (256, 3), (0, 0), (512, 5)])
def test_cta_pair_dense_cluster(k_chunk, split_k):
    wl = _dense_cluster()
    F = run_gpu(wl, "tc_split16", flags_extra=kde.FLAG_CTA_PAIR, k_chunk=k_chunk, split_k=split_k)
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, oracle.GAUSSIAN)
    assert rel_linf(F, ref) <= TOL_SPLIT


def test_cta_pair_batched_matches_single():
    wls = [workloads.random_points(420 + k, 2000 + 500 * k, 4000.0, 10.0, 200 + 40 * k,
                                   300 - 30 * k, 35.0, oracle.GAUSSIAN) for k in range(5)]
    insts = [dict(points=torch.as_tensor(wl.xy, dtype=torch.float64, device="cuda"),
                  weights=torch.as_tensor(wl.w, dtype=torch.float32, device="cuda"),
                  origin=wl.origin, cell=wl.cell, nx=wl.nx, ny=wl.ny, h=wl.h, kernel="gaussian")
             for wl in wls]
    outs = kde.grid_batched(insts, flags=kde.FLAG_SYNC | kde.FLAG_CTA_PAIR, split_k=2)
    for wl, d, F in zip(wls, insts, outs):
        alone = kde.grid(d["points"], d["weights"], wl.origin, wl.cell, wl.nx, wl.ny, wl.h,
                         "gaussian", flags=kde.FLAG_SYNC | kde.FLAG_CTA_PAIR, split_k=2)
        assert torch.equal(F, alone)
        ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h,
                              oracle.GAUSSIAN)
        assert rel_linf(F.cpu().numpy(), ref) <= TOL_SPLIT


@pytest.mark.parametrize("path,flags", [
    ("auto", 0), ("tc_split16", kde.FLAG_CTA_PAIR), ("tc_split16", kde.FLAG_ONE_CTA),
    ("tc_fp16", kde.FLAG_ONE_CTA), ("tc_fp16", kde.FLAG_CTA_PAIR), ("tc_split16", kde.FLAG_SKIP_ZERO)],
    ids=["auto", "split-pair", "split-one-cta", "fp16-one-cta", "fp16-pair", "split-sparse"])
def test_signed_weights_match_oracle(path, flags):
    """Weights of both signs (a density minus another, Eq. 7 with signed w):
    every tensor-core variant, and AUTO, match the oracle; the error is
    normalised by max |F|."""
    wl = workloads.random_points(402, 6001, 5000.0, 12.5, 300, 280, 40.0, oracle.GAUSSIAN)
    rng = np.random.default_rng(402)
    wl.w = (rng.uniform(0.5, 2.0, wl.n) * np.where(rng.random(wl.n) < 0.4, -1.0, 1.0)).astype(
        np.float32)
    F = run_gpu(wl, path, flags_extra=flags)
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, oracle.GAUSSIAN)
    assert np.min(ref) < 0 < np.max(ref)
    assert rel_linf(F, ref) <= TOL.get(path, TOL_SPLIT)


def test_all_negative_weights_flip_the_density():
    wl = workloads.random_points(403, 2500, 3000.0, 10.0, 256, 300, 35.0, oracle.GAUSSIAN)
    neg = workloads.random_points(403, 2500, 3000.0, 10.0, 256, 300, 35.0, oracle.GAUSSIAN)
    neg.w = -wl.w
    F = run_gpu(wl, "auto")
    Fn = run_gpu(neg, "auto")
    np.testing.assert_array_equal(Fn, -F)
