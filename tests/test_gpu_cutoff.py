"""Parity of the binned cutoff path (path c, compact kernels) with the FP64
oracle, through the C ABI, on the GPU (FP32: 1e-6 relative L-inf)."""
import numpy as np
import pytest

import oracle
import workloads
from kde_testutil import TOL_FP32, clear_of_support_edge, rel_linf, sample_cells

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2004_13653_gb300 as kde  # noqa: E402

COMPACT = [k for k in range(8) if k != oracle.GAUSSIAN]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kde.load(build_if_stale=True)


def run_gpu(wl, kid, path="cutoff", weights=True):
    pts = torch.as_tensor(np.ascontiguousarray(wl.xy), dtype=torch.float64, device="cuda")
    w = torch.as_tensor(wl.w, dtype=torch.float32, device="cuda") if weights else None
    out = kde.grid(pts, w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, kid, path=path,
                   flags=kde.FLAG_SYNC)
    return out.cpu().numpy()


@pytest.mark.parametrize("kid", COMPACT, ids=[oracle.KERNEL_NAMES[k] for k in COMPACT])
def test_all_compact_kernels_ragged(kid):
    """Ragged 16x16 output blocks on both axes (4-cell sort bins), weights
    U(0.5, 2), points partly outside the grid (some beyond reach, some within
    a bandwidth)."""
    wl = workloads.random_points(500 + kid, 2500, 3000.0, 10.0, 300, 150, 35.0, kid)
    if kid == oracle.UNIFORM:
        wl = clear_of_support_edge(wl, radial=False)
    F = run_gpu(wl, kid)
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, kid)
    assert rel_linf(F, ref) <= TOL_FP32


@pytest.mark.parametrize("kid", [oracle.EPANECHNIKOV, oracle.TRICUBE])
def test_wide_bandwidth_many_bins_in_reach(kid):
    """h = 70 cells (16-cell sort bins): each output block reads the points of
    a 10 x 10 window of sort bins."""
    wl = workloads.random_points(510 + kid, 3000, 700.0, 5.0, 128, 96, 350.0, kid)
    F = run_gpu(wl, kid)
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, kid)
    assert rel_linf(F, ref) <= TOL_FP32


@pytest.mark.parametrize("h_cells", [1.5, 5.0, 6.5, 12.0, 16.5, 30.0])
@pytest.mark.parametrize("kid", [oracle.EPANECHNIKOV, oracle.RADIAL + oracle.QUARTIC],
                         ids=["epanechnikov", "radial_quartic"])
def test_every_sort_bin_side(h_cells, kid):
    """Bandwidths on both sides of each change of sort-bin side (4 cells up
    to 6 h/cell, 8 up to 16, 16 beyond), clustered points on a ragged grid:
    the points an output block reads must include every point within a
    bandwidth of its cells."""
    cell = 10.0
    wl = workloads.random_points(540 + int(h_cells * 10), 3000, 2400.0, cell, 230, 170,
                                 h_cells * cell, kid % oracle.RADIAL)
    wl.local[:1000] = wl.local[:1000] * 0.1 + 1100.0  # a dense cluster
    F = run_gpu(wl, kid)
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, kid)
    assert rel_linf(F, ref) <= TOL_FP32


def test_config2_epanechnikov_sampled_and_vs_simt():
    wl = workloads.config2(kernel=oracle.EPANECHNIKOV)
    F = run_gpu(wl, oracle.EPANECHNIKOV)
    cells = sample_cells(F, 256, seed=21)
    ref = oracle.kde_cells(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h,
                           oracle.EPANECHNIKOV, cells)
    assert rel_linf(F.reshape(-1)[cells], ref) <= TOL_FP32
    S = run_gpu(wl, oracle.EPANECHNIKOV, path="simt")
    assert rel_linf(F, S) <= 2 * TOL_FP32


def test_bitwise_reproducible():
    wl = workloads.config2(kernel=oracle.QUARTIC, n_traj=400)
    a = run_gpu(wl, oracle.QUARTIC)
    b = run_gpu(wl, oracle.QUARTIC)
    assert np.array_equal(a, b)


def test_all_points_out_of_reach_give_zeros():
    wl = workloads.random_points(520, 100, 1000.0, 10.0, 50, 50, 20.0, oracle.EPANECHNIKOV)
    wl.local[:] += 1e6
    F = run_gpu(wl, oracle.EPANECHNIKOV)
    assert not F.any()


def test_single_point_and_auto_path():
    wl = workloads.random_points(521, 1, 200.0, 10.0, 20, 20, 30.0, oracle.TRIWEIGHT)
    wl.local[:] = [[101.0, 99.0]]
    F = run_gpu(wl, oracle.TRIWEIGHT, path="auto")
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, oracle.TRIWEIGHT)
    assert rel_linf(F, ref) <= TOL_FP32


RADIAL_COMPACT = [oracle.RADIAL + k for k in COMPACT]


@pytest.mark.parametrize("kid", RADIAL_COMPACT,
                         ids=["radial_" + oracle.KERNEL_NAMES[k - oracle.RADIAL]
                              for k in RADIAL_COMPACT])
def test_radial_kernels_ragged(kid):
    """Radial variants on the disk (cutoff path, AUTO): ragged bins, weights,
    points partly outside the grid."""
    wl = workloads.random_points(530 + kid, 2500, 3000.0, 10.0, 300, 150, 35.0, kid)
    if kid == oracle.RADIAL + oracle.UNIFORM:
        wl = clear_of_support_edge(wl, radial=True)
    F = run_gpu(wl, kid, path="auto")
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, kid)
    assert rel_linf(F, ref) <= TOL_FP32


def test_radial_wide_bandwidth_sampled():
    """1M lane points on 1024^2, h = 150 m (3 cells), radial Epanechnikov,
    sampled cells."""
    kid = oracle.RADIAL + oracle.EPANECHNIKOV
    wl = workloads.config2(kernel=kid)
    F = run_gpu(wl, kid)
    cells = sample_cells(F, 256, seed=23)
    ref = oracle.kde_cells(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, kid, cells)
    assert rel_linf(F.reshape(-1)[cells], ref) <= TOL_FP32


def test_radial_gaussian_is_the_gaussian_and_simt_rejects_radial():
    wl = workloads.config1()
    a = run_gpu(wl, oracle.GAUSSIAN, path="tc_split16")
    b = run_gpu(wl, oracle.RADIAL + oracle.GAUSSIAN, path="tc_split16")
    np.testing.assert_array_equal(a, b)
    with pytest.raises(RuntimeError):
        run_gpu(wl, oracle.RADIAL + oracle.EPANECHNIKOV, path="simt")


@pytest.mark.parametrize("kid", COMPACT, ids=[oracle.KERNEL_NAMES[k] for k in COMPACT])
def test_all_compact_kernels_sort_bins_of_8(kid):
    """h = 12 cells (8-cell sort bins) for every compact kernel, ragged grid."""
    wl = workloads.random_points(560 + kid, 2000, 2600.0, 10.0, 230, 170, 120.0, kid)
    if kid == oracle.UNIFORM:
        wl = clear_of_support_edge(wl, radial=False)
    F = run_gpu(wl, kid)
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, kid)
    assert rel_linf(F, ref) <= TOL_FP32


@pytest.mark.parametrize("kid", [oracle.EPANECHNIKOV, oracle.RADIAL + oracle.TRIWEIGHT],
                         ids=["epanechnikov", "radial_triweight"])
def test_points_on_sort_bin_edges_far_from_origin(kid):
    """A 20,000-cell-wide grid (coordinates up to 10^4 bandwidths, where the
    FP32 bin keys are coarsest) with points exactly on sort-bin edges, one
    cell either side of them and at random, near the far end: the points a
    block reads must still include every point within a bandwidth of its
    cells."""
    rng = np.random.default_rng(570 + kid)
    cell, nx, ny, h = 10.0, 20000, 48, 20.0  # h = 2 cells: 4-cell sort bins
    k = rng.integers(4900, 5000, 400).astype(np.float64)
    edges = k * 4 * cell
    xs = np.concatenate([edges, edges + cell, edges - cell, rng.uniform(19_500 * cell, nx * cell, 400)])
    ys = rng.uniform(0.0, ny * cell, xs.size)
    wl = workloads.random_points(571, xs.size, 1.0, cell, nx, ny, h, kid % oracle.RADIAL)
    wl.local[:] = np.stack([xs, ys], axis=1)
    F = run_gpu(wl, kid)
    # the cells around the first 300 edge points (and their neighbours one cell off)
    ci = np.floor(xs[:300] / cell).astype(np.int64)
    cj = np.floor(ys[:300] / cell).astype(np.int64)
    cells = np.unique(np.concatenate([
        np.clip(cj + dj, 0, ny - 1) * nx + np.clip(ci + di, 0, nx - 1)
        for di in range(-3, 4) for dj in (-1, 0, 1)]))
    ref = oracle.kde_cells(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, kid, cells)
    assert np.max(ref) > 0
    assert rel_linf(F.reshape(-1)[cells], ref) <= TOL_FP32


def _heavy_cluster(seed, kid, h_cells, n=30_000, dense=20_000):
    """n points on a ragged 150 x 120 grid of 10 m cells, `dense` of them in a
    180 m square that straddles output-block borders: the blocks there have
    4096 points or more within reach, and for supports of up to 6 cells they
    are computed as four 4-row slices."""
    cell = 10.0
    wl = workloads.random_points(seed, n, 1600.0, cell, 150, 120, h_cells * cell, kid % oracle.RADIAL)
    rng = np.random.default_rng(seed + 1)
    wl.local[:dense] = rng.uniform([470.0, 310.0], [650.0, 490.0], size=(dense, 2))
    return wl


@pytest.mark.parametrize("h_cells", [1.0, 3.5, 12.0, 30.0])
@pytest.mark.parametrize("kid", [oracle.EPANECHNIKOV, oracle.RADIAL + oracle.TRICUBE],
                         ids=["epanechnikov", "radial_tricube"])
def test_heavy_blocks_in_row_slices(h_cells, kid):
    """Heavy blocks next to light ones against the oracle on the whole grid:
    split into row slices, each with its own range of sort bins, at h = 1
    and 3.5 cells (4-cell sort bins); whole at 12 and 30 cells (8- and
    16-cell sort bins)."""
    wl = _heavy_cluster(585 + int(h_cells), kid, h_cells)
    F = run_gpu(wl, kid)
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, kid)
    assert rel_linf(F, ref) <= TOL_FP32


def test_heavy_blocks_reproducible_and_same_in_a_batch():
    """A block's split into slices depends only on its own point count: the
    result is the same bits run after run and inside a batch."""
    kid = oracle.QUARTIC
    wl = _heavy_cluster(590, kid, 3.0)
    other = workloads.random_points(591, 5000, 900.0, 7.5, 97, 61, 20.0, oracle.EPANECHNIKOV)
    a = run_gpu(wl, kid)
    assert np.array_equal(a, run_gpu(wl, kid))

    def inst(x, k):
        return dict(points=torch.as_tensor(x.xy, dtype=torch.float64, device="cuda"),
                    weights=torch.as_tensor(x.w, dtype=torch.float32, device="cuda"),
                    origin=x.origin, cell=x.cell, nx=x.nx, ny=x.ny, h=x.h, kernel=k)
    outs = kde.grid_batched([inst(other, oracle.EPANECHNIKOV), inst(wl, kid)], flags=kde.FLAG_SYNC)
    assert np.array_equal(outs[1].cpu().numpy(), a)
    assert np.array_equal(outs[0].cpu().numpy(), run_gpu(other, oracle.EPANECHNIKOV))


def _wide_grid(seed, n_side, cell, centre):
    """60,000 points: two thirds uniform over an n_side^2 grid, one third in
    a cluster of sigma 30 m, at h = 2 cells (4-cell sort bins)."""
    rng = np.random.default_rng(seed)
    kid = oracle.EPANECHNIKOV
    wl = workloads.random_points(seed, 60_000, 1.0, cell, n_side, n_side, 2.0 * cell, kid)
    wl.local[:40_000] = rng.uniform(0.0, n_side * cell, size=(40_000, 2))
    wl.local[40_000:] = rng.normal(np.asarray(centre) * n_side * cell, 30.0, size=(20_000, 2))
    return wl


@pytest.mark.parametrize("nx,ny", [(68, 60), (64, 64), (1028, 4), (1020, 1028), (262148, 4)],
                         ids=["255-bins", "256-bins", "257-bins", "65535-bins", "65537-bins"])
def test_sort_pass_count_boundaries(nx, ny):
    """Grids whose 4-cell sort bins number 255, 256, 257, 65535 and 65537
    (1024^2's 65536 is covered elsewhere): valid keys of 8, 8, 9, 16 and 17
    bits, the padding key fitting the top digit or taking the bucket above
    the digits, on either side of every change in the number of passes.
    Points over and around the grid, a share beyond reach; n not a multiple
    of the sort's chunk.  Against the oracle on every cell of the small grids
    and on sampled cells of the large ones."""
    kid = oracle.EPANECHNIKOV
    cell = 10.0
    rng = np.random.default_rng(nx + 7 * ny)
    wl = workloads.random_points(nx + ny, 20_003, 1.0, cell, nx, ny, 2.0 * cell, kid)
    W, H = nx * cell, ny * cell
    wl.local[:] = np.stack([rng.uniform(-0.2 * W, 1.2 * W, wl.n),
                            rng.uniform(-0.2 * H - 50.0, 1.2 * H + 50.0, wl.n)], 1)
    F = run_gpu(wl, kid)
    if nx * ny <= 5000:
        ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, kid)
        assert rel_linf(F, ref) <= TOL_FP32
    else:
        cells = sample_cells(F, 512, seed=nx)
        ref = oracle.kde_cells(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, kid, cells)
        assert np.max(ref) > 0
        assert rel_linf(F.reshape(-1)[cells], ref) <= TOL_FP32


def test_three_radix_passes_and_the_marker_bucket_on_a_16384_square_grid():
    """16384^2 cells at h = 2 cells: 4096^2 = 2^24 sort bins of 4 cells.  The
    valid keys take 24 bits (three 8-bit passes, the last writing the
    permuted points); the key of padding, total_bins = 2^24, has the 25th bit
    and sorts in the bucket above the digits in every pass.  The gather takes
    a million output blocks; sampled cells around the densest one and
    elsewhere against the oracle."""
    kid = oracle.EPANECHNIKOV
    wl = _wide_grid(599, 16384, 10.0, (0.7, 0.2))
    F = run_gpu(wl, kid)
    assert F.shape == (16384, 16384)
    cells = sample_cells(F, 512, seed=600)
    ref = oracle.kde_cells(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, kid, cells)
    assert np.max(ref) > 0
    assert rel_linf(F.reshape(-1)[cells], ref) <= TOL_FP32


def test_four_radix_passes_on_a_batch_of_two_16384_square_grids():
    """Two 16384^2 instances in one batch share one sort over 2^25 bins: keys
    of 25 bits run all four passes (the padding key 2^25 then fits the top
    digit).  Each instance is checked at sampled cells against the oracle and
    equals its own single call bit for bit."""
    kid = oracle.EPANECHNIKOV
    wls = [_wide_grid(601, 16384, 10.0, (0.3, 0.8)), _wide_grid(602, 16384, 10.0, (0.5, 0.5))]
    insts = []
    for wl in wls:
        insts.append(dict(points=torch.as_tensor(wl.xy, dtype=torch.float64, device="cuda"),
                          weights=torch.as_tensor(wl.w, dtype=torch.float32, device="cuda"),
                          origin=wl.origin, cell=wl.cell, nx=wl.nx, ny=wl.ny, h=wl.h,
                          kernel=kid))
    outs = kde.grid_batched(insts, flags=kde.FLAG_SYNC)
    for k, (wl, F) in enumerate(zip(wls, outs)):
        Fh = F.cpu().numpy()
        cells = sample_cells(Fh, 256, seed=603 + k)
        ref = oracle.kde_cells(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, kid, cells)
        assert np.max(ref) > 0
        assert rel_linf(Fh.reshape(-1)[cells], ref) <= TOL_FP32
        del Fh
    alone = run_gpu(wls[1], kid)
    assert np.array_equal(outs[1].cpu().numpy(), alone)
