"""Parity of the FP32 SIMT path (path a) and the FP64 prep steps with the
oracle, through the C ABI, on the GPU."""
import numpy as np
import pytest

import oracle
import workloads
from kde_testutil import TOL_FP32, rel_linf, sample_cells

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2004_13653_gb300 as kde  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kde.load(build_if_stale=True)


def _dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def run_gpu(wl, path="simt", kernel=None, weights=True, **kw):
    pts = _dev(wl.xy, torch.float64)
    w = _dev(wl.w, torch.float32) if weights else None
    out = kde.grid(pts, w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h,
                   wl.kernel if kernel is None else kernel, path=path, flags=kde.FLAG_SYNC, **kw)
    return out.cpu().numpy()


def test_config1_full_grid():
    wl = workloads.config1()
    F = run_gpu(wl)
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, wl.kernel)
    assert rel_linf(F, ref) <= TOL_FP32


@pytest.mark.parametrize("kid", range(8), ids=oracle.KERNEL_NAMES)
def test_all_kernels_ragged_tiles(kid):
    """Several 128x64 tiles with ragged edges, n not a multiple of the point
    tile, non-unit weights, points partly outside the grid."""
    wl = workloads.random_points(200 + kid, 1000, 3000.0, 10.0, 300, 150, 35.0, kid)
    F = run_gpu(wl)
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, kid)
    assert rel_linf(F, ref) <= TOL_FP32


@pytest.mark.parametrize("kernel", [oracle.GAUSSIAN, oracle.EPANECHNIKOV])
def test_config2_sampled(kernel):
    wl = workloads.config2(kernel=kernel)
    F = run_gpu(wl)
    cells = sample_cells(F, 256, seed=kernel)
    ref = oracle.kde_cells(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, kernel, cells)
    assert rel_linf(F.reshape(-1)[cells], ref) <= TOL_FP32


@pytest.mark.parametrize("split_k", [1, 3, 7])
def test_split_k_counts_agree(split_k):
    wl = workloads.random_points(300, 5000, 2000.0, 20.0, 100, 100, 60.0, oracle.GAUSSIAN)
    F = run_gpu(wl, split_k=split_k)
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, wl.kernel)
    assert rel_linf(F, ref) <= TOL_FP32


def test_unit_weights_as_null():
    wl = workloads.config1()
    F = run_gpu(wl, weights=False)
    ref = oracle.kde_grid(wl.xy, None, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, wl.kernel)
    assert rel_linf(F, ref) <= TOL_FP32


def test_single_cell_and_single_point():
    wl = workloads.random_points(301, 1, 100.0, 10.0, 1, 1, 50.0, oracle.GAUSSIAN)
    wl.local[:] = [[3.0, 4.0]]
    F = run_gpu(wl)
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, 1, 1, wl.h, wl.kernel)
    assert F.shape == (1, 1)
    assert rel_linf(F, ref) <= TOL_FP32


def test_empty_input_writes_zeros():
    out = torch.full((5, 7), 3.0, device="cuda")
    pts = torch.zeros((0, 2), dtype=torch.float64, device="cuda")
    kde.grid(pts, None, (0.0, 0.0), 1.0, 7, 5, 2.0, "gaussian", out=out, path="simt",
             flags=kde.FLAG_SYNC)
    assert torch.count_nonzero(out).item() == 0


def test_host_buffers_through_plain_entry():
    """kde_grid with host (numpy) points and output: staged through the workspace."""
    wl = workloads.config1()
    out = np.zeros((wl.ny, wl.nx), dtype=np.float32)
    xy = np.ascontiguousarray(wl.xy)
    kde.grid_simple(xy, np.ascontiguousarray(wl.w), wl.origin, wl.cell, wl.nx, wl.ny, wl.h,
                    wl.kernel, out)
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, wl.kernel)
    assert rel_linf(out, ref) <= 1e-5  # AUTO path


def test_plain_entry_runs_on_the_set_stream():
    """kde_set_stream: the points reach their device buffer on a side stream
    only after a ~0.1 s spin; kde_grid on that stream reads them in order and
    matches the oracle (on the legacy stream it would race the spin, because
    torch's streams do not synchronise with it).  Another thread, which has
    set no stream, still runs on the legacy stream."""
    import threading
    wl = workloads.config1()
    src = _dev(wl.xy, torch.float64)
    pts = torch.zeros_like(src)
    w = _dev(wl.w, torch.float32)
    out = torch.full((wl.ny, wl.nx), 7.0, device="cuda")
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, wl.kernel)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    try:
        kde.set_stream(side)
        with torch.cuda.stream(side):
            torch.cuda._sleep(200_000_000)
            pts.copy_(src)
        kde.grid_simple(pts, w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, wl.kernel, out)
        assert side.query()  # kde_grid waited for its stream
        assert rel_linf(out.cpu().numpy(), ref) <= 1e-5

        other = torch.full_like(out, 7.0)
        torch.cuda.synchronize()
        errs = []

        def worker():
            try:
                kde.grid_simple(pts, w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, wl.kernel,
                                other)
            except Exception as e:  # reported below, on the test's thread
                errs.append(e)
        t = threading.Thread(target=worker)
        t.start()
        t.join()
        assert not errs
        assert rel_linf(other.cpu().numpy(), ref) <= 1e-5
    finally:
        kde.set_stream(None)
    torch.cuda.synchronize()
    out.fill_(7.0)
    kde.grid_simple(pts, w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, wl.kernel, out)
    assert rel_linf(out.cpu().numpy(), ref) <= 1e-5


def test_plain_entry_with_host_buffers_on_a_set_stream():
    """Host (numpy) points, weights and output through kde_grid while a side
    stream is set: the copies go through the workspace on that stream and the
    call still returns the finished density, equal to the oracle's."""
    wl = workloads.config1()
    side = torch.cuda.Stream()
    out = np.full((wl.ny, wl.nx), np.nan, dtype=np.float32)
    try:
        kde.set_stream(side)
        kde.grid_simple(np.ascontiguousarray(wl.xy), np.ascontiguousarray(wl.w), wl.origin,
                        wl.cell, wl.nx, wl.ny, wl.h, wl.kernel, out)
    finally:
        kde.set_stream(None)
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, wl.kernel)
    assert np.isfinite(out).all()
    assert rel_linf(out, ref) <= 1e-5  # AUTO path


def test_nonfinite_coordinate_reported():
    wl = workloads.config1()
    xy = wl.xy.copy()
    xy[17, 1] = np.nan
    with pytest.raises(kde.KDEError) as e:
        kde.grid(_dev(xy, torch.float64), None, wl.origin, wl.cell, wl.nx, wl.ny, wl.h,
                 "gaussian", path="simt", flags=kde.FLAG_SYNC)
    assert e.value.code == kde.KDE_EDATA


def test_mercator_matches_oracle():
    wl = workloads.config2()
    ll, corner, lat0 = wl.lonlat()
    got = kde.project_mercator(_dev(ll, torch.float64), lat0)
    torch.cuda.synchronize()
    ref = oracle.mercator(ll, lat0)
    np.testing.assert_allclose(got.cpu().numpy(), ref, rtol=0, atol=1e-6)


@pytest.mark.parametrize("lat0", [-45.0, 0.0, 31.35, 60.0, 80.0])
def test_mercator_series_and_closed_form(lat0):
    """Latitudes within and beyond the range where the projection uses its
    series about lat0 (the rest take the closed form), both hemispheres, high
    latitude; 1e-6 m of the oracle everywhere."""
    rng = np.random.default_rng(int(lat0 * 10) + 1000)
    lat = lat0 + np.concatenate([rng.uniform(-0.5, 0.5, 4000), rng.uniform(-3.0, 3.0, 1000),
                                 [0.0, 0.57, -0.57]])
    lat = np.clip(lat, -85.0, 85.0)
    ll = np.stack([rng.uniform(-180.0, 180.0, lat.size), lat], axis=1)
    got = kde.project_mercator(_dev(ll, torch.float64), lat0)
    torch.cuda.synchronize()
    ref = oracle.mercator(ll, lat0)
    np.testing.assert_allclose(got.cpu().numpy(), ref, rtol=0, atol=1e-6)


def test_lonlat_pipeline_matches_oracle():
    """Project on the GPU, then the density; the oracle projects on its own."""
    wl = workloads.config1()
    ll, corner, lat0 = wl.lonlat()
    xy_dev = kde.project_mercator(_dev(ll, torch.float64), lat0)
    origin = oracle.mercator([corner], lat0)[0]
    F = kde.grid(xy_dev, _dev(wl.w, torch.float32), origin, wl.cell, wl.nx, wl.ny, wl.h,
                 "gaussian", path="simt", flags=kde.FLAG_SYNC).cpu().numpy()
    xy_ref = oracle.mercator(ll, lat0)
    ref = oracle.kde_grid(xy_ref, wl.w, origin, wl.cell, wl.nx, wl.ny, wl.h, oracle.GAUSSIAN)
    assert rel_linf(F, ref) <= TOL_FP32
