"""Parity of the paper's binned estimator (Sec. IV-B: Algorithm 3 count matrix,
Eq. InterX/InterY interpolation, Eq. 7 convolution) with the FP64 oracle,
through the C ABI, on the GPU.  Counts are compared bit for bit; the
convolution to 1e-6 relative L-inf (FP32)."""
import math

import numpy as np
import pytest

import oracle
import workloads
from kde_testutil import TOL_FP32, rel_linf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2004_13653_gb300 as kde  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kde.load(build_if_stale=True)


def auto_window(kid, h, cell):
    a = math.ceil(4.0 * h / cell) if kid == oracle.GAUSSIAN else math.floor(h / cell)
    return 2 * min(a, 127) + 1


def run(xy, offsets, origin, cell, nx, ny, h, kid, window=0, interpolate=True):
    pts = torch.as_tensor(np.ascontiguousarray(xy), dtype=torch.float64, device="cuda")
    off = None if offsets is None else torch.as_tensor(np.asarray(offsets, np.int64),
                                                       device="cuda")
    F, C, added = kde.grid_binned(pts, off, origin, cell, nx, ny, h, kid, window, interpolate)
    torch.cuda.synchronize()
    return F.cpu().numpy(), C.cpu().numpy(), added


def check(xy, offsets, origin, cell, nx, ny, h, kid, window=0, interpolate=True):
    n = xy.shape[0]
    F, C, added = run(xy, offsets, origin, cell, nx, ny, h, kid, window, interpolate)
    off = np.array([0, n], np.int64) if offsets is None else offsets
    C_ref, added_ref = oracle.count_matrix(xy, off, origin, cell, nx, ny, interpolate)
    assert added == added_ref
    np.testing.assert_array_equal(C, C_ref)
    win = window or auto_window(kid, h, cell)
    F_ref = oracle.convolve(C_ref, cell, h, kid, win, n)
    if np.max(np.abs(F_ref)) > 0:
        assert rel_linf(F, F_ref) <= TOL_FP32
    else:
        assert not np.any(F)
    return F, C, added


@pytest.mark.parametrize("interpolate", [False, True])
def test_config2_counts_and_convolution(interpolate):
    """1M fixes of 2000 lane trajectories on the 1024^2 grid, Gaussian."""
    wl = workloads.config2()
    _, C, added = check(wl.xy, wl.offsets, wl.origin, wl.cell, wl.nx, wl.ny, wl.h,
                        oracle.GAUSSIAN, interpolate=interpolate)
    assert (added > 0) == interpolate
    inside = np.all((wl.local >= 0) & (wl.local < wl.box), axis=1).sum()
    assert int(C.sum()) == inside + added


def test_sparse_fixes_long_gaps_ragged_trajectories():
    """Every 25th fix (gaps of tens of cells), trajectories of ragged length,
    some fixes outside the grid (no interpolation across them)."""
    wl = workloads.config2(seed=1012, n_traj=300, fixes=500, kernel=oracle.EPANECHNIKOV)
    xy = wl.xy[::25].copy()
    n = xy.shape[0]
    rng = np.random.default_rng(7)
    cuts = np.sort(rng.choice(np.arange(1, n), size=97, replace=False))
    offsets = np.concatenate([[0], cuts, [n]]).astype(np.int64)
    xy[rng.choice(n, 40, replace=False)] += 60_000.0   # pushed off the grid
    for kid in (oracle.EPANECHNIKOV, oracle.UNIFORM, oracle.COSINE):
        _, _, added = check(xy, offsets, wl.origin, wl.cell, wl.nx, wl.ny, 400.0, kid)
        assert added > 10 * n


@pytest.mark.parametrize("kid", range(8), ids=oracle.KERNEL_NAMES)
def test_all_kernels_ragged_grid(kid):
    """A 300 x 170 grid (ragged against the 128-wide and 64-high tiles), one
    trajectory (NULL offsets), every Table 1 kernel."""
    wl = workloads.random_points(600 + kid, 4000, 3000.0, 10.0, 300, 170, 45.0, kid)
    check(wl.xy, None, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, kid)


def test_window_extremes():
    """window 1 (only the centre weight k(0)^2) and the 255 maximum."""
    wl = workloads.random_points(620, 3000, 2000.0, 8.0, 260, 200, 30.0, oracle.GAUSSIAN)
    F, C, _ = check(wl.xy, None, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, oracle.GAUSSIAN,
                    window=1, interpolate=False)
    k0 = 1.0 / math.sqrt(2.0 * math.pi)
    n = wl.xy.shape[0]
    np.testing.assert_allclose(F, C * (k0 * k0 / (n * wl.h * wl.h)), rtol=1e-6, atol=0)
    check(wl.xy, None, wl.origin, wl.cell, wl.nx, wl.ny, 400.0, oracle.GAUSSIAN, window=255)


def test_empty_and_all_outside():
    origin = workloads.FALSE_ORIGIN
    F, C, added = run(np.zeros((0, 2)), None, origin, 10.0, 70, 33, 25.0, oracle.QUARTIC)
    assert added == 0 and not C.any() and not F.any()
    xy = np.array(origin) + np.array([[-5.0, 3.0], [800.0, 5.0], [5.0, 400.0]])
    F, C, added = run(xy, None, origin, 10.0, 70, 33, 25.0, oracle.QUARTIC)
    assert added == 0 and not C.any() and not F.any()


def test_invalid_arguments():
    pts = torch.zeros(8, dtype=torch.float64, device="cuda")
    origin = workloads.FALSE_ORIGIN
    with pytest.raises(RuntimeError):
        kde.grid_binned(pts, None, origin, 10.0, 16, 16, 25.0, oracle.GAUSSIAN, window=4)
    with pytest.raises(RuntimeError):
        kde.grid_binned(pts, None, origin, 10.0, 16, 16, 25.0, oracle.GAUSSIAN, window=257)
    with pytest.raises(RuntimeError):
        kde.grid_binned(pts.cpu(), None, origin, 10.0, 16, 16, 25.0, oracle.GAUSSIAN,
                        stream=torch.cuda.current_stream())


def test_binned_vs_direct_sum_on_dense_grid():
    """The binned estimator approximates the direct sum; with h = 8 cells, no
    interpolation and three Gaussian clusters well inside the grid, the
    difference is the binning error, well below 10% of the peak (a wrong
    normalisation or a transposed stencil is not)."""
    rng = np.random.default_rng(630)
    centres = np.array([[800.0, 800.0], [1700.0, 1200.0], [1300.0, 1900.0]])
    local = centres[rng.integers(0, 3, 20000)] + rng.normal(0.0, 150.0, (20000, 2))
    origin = workloads.FALSE_ORIGIN
    xy = local + np.array(origin)
    F, _, _ = check(xy, None, origin, 10.0, 256, 256, 80.0, oracle.GAUSSIAN, interpolate=False)
    D = oracle.kde_grid(xy, np.ones(20000, np.float32), origin, 10.0, 256, 256, 80.0,
                        oracle.GAUSSIAN)
    err = rel_linf(F, D)
    print(f"binned vs direct sum: {err:.3e}")
    assert err < 0.1


@pytest.mark.parametrize("cell", [10.0, 24.4140625, 7.3])
def test_fixes_on_and_next_to_cell_edges(cell):
    """Fixes exactly on cell edges (o + k cell in FP64) and one ulp either
    side of them, along x and y, with an origin and a cell that are not
    powers of two: the cell index must be the floor of the correctly rounded
    FP64 division in every case (the kernel decides most cells with a
    multiply and divides only next to an edge)."""
    rng = np.random.default_rng(int(cell * 1000))
    origin = (512_345.678, 4_401_234.5)
    nx, ny = 300, 200
    k = rng.integers(0, nx, 3000).astype(np.float64)
    m = rng.integers(0, ny, 3000).astype(np.float64)
    ex = origin[0] + k * cell
    ey = origin[1] + m * cell
    xs = np.concatenate([ex, np.nextafter(ex, -np.inf), np.nextafter(ex, np.inf), ex + 0.3 * cell])
    ys = np.concatenate([ey + 0.5 * cell, ey, np.nextafter(ey, np.inf), np.nextafter(ey, -np.inf)])
    xy = np.stack([xs, ys], axis=1)
    check(xy, None, origin, cell, nx, ny, 3.0 * cell, oracle.EPANECHNIKOV, interpolate=False)
