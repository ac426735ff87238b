"""Block-sparse skipping on the tensor-core path (KDE_FLAG_SKIP_ZERO): the
result must stay within the path's tolerance of the FP64 oracle (split-FP16
1e-5, FP16 2e-3) and agree with the dense contraction to rounding, since the
skipped operands are exactly zero in FP16.  Cases: ragged grids, points
outside the grid within reach, clustered points (tiles cut into many pieces),
wide bandwidths (reach over several bins), batches mixed with the cutoff
path, empty work lists, graph capture."""
import numpy as np
import pytest

import oracle
import workloads
from kde_testutil import TOL_FP16, TOL_SPLIT, rel_linf, sample_cells

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2004_13653_gb300 as kde  # noqa: E402

TOL = {"tc_fp16": TOL_FP16, "tc_split16": TOL_SPLIT}
# sparse vs dense: the same products summed in another order (the points are
# sorted), so only the FP32 accumulation's rounding differs
SAME = {"tc_fp16": 1e-5, "tc_split16": 2e-6}
SPARSE = kde.FLAG_SKIP_ZERO | kde.FLAG_SYNC


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kde.load(build_if_stale=True)


def dev(wl):
    pts = torch.as_tensor(np.ascontiguousarray(wl.xy), dtype=torch.float64, device="cuda")
    w = torch.as_tensor(wl.w, dtype=torch.float32, device="cuda")
    return pts, w


def run(wl, path, flags):
    pts, w = dev(wl)
    out = kde.grid(pts, w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, "gaussian", path=path,
                   flags=flags)
    return out.cpu().numpy()


@pytest.mark.parametrize("path", ["tc_split16", "tc_fp16"])
def test_ragged_grid_points_outside(path):
    """700 x 300 grid (ragged 256-tiles), points from -10% to 110% of the box:
    some outside within reach, some beyond it."""
    wl = workloads.random_points(700, 6001, 9000.0, 12.5, 700, 300, 30.0, oracle.GAUSSIAN)
    F = run(wl, path, SPARSE)
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, oracle.GAUSSIAN)
    assert rel_linf(F, ref) <= TOL[path]
    D = run(wl, path, kde.FLAG_SYNC | kde.FLAG_CTA_PAIR)
    assert rel_linf(F, D) <= SAME[path]


@pytest.mark.parametrize("h", [60.0, 400.0])
def test_wide_and_narrow_bandwidth(h):
    """h = 4.8 cells (reach inside one bin) and h = 32 cells (reach of ~240
    cells: a bin is within reach of up to four tiles per axis)."""
    wl = workloads.random_points(710, 8000, 8000.0, 12.5, 640, 640, h, oracle.GAUSSIAN)
    F = run(wl, "tc_split16", SPARSE)
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, oracle.GAUSSIAN)
    assert rel_linf(F, ref) <= TOL_SPLIT


def test_clustered_config3_shape_sampled():
    """The 20M-point mixture's generator at 2M points on 1024^2: port
    clusters put hundreds of thousands of points into a few tiles, which the
    work list cuts into many pieces."""
    wl = workloads.config3(n_traj=4000, grid=1024)
    F = run(wl, "tc_split16", SPARSE)
    cells = sample_cells(F, 512, seed=31)
    ref = oracle.kde_cells(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h,
                           oracle.GAUSSIAN, cells)
    assert rel_linf(F.reshape(-1)[cells], ref) <= TOL_SPLIT
    D = run(wl, "tc_split16", kde.FLAG_SYNC)
    assert rel_linf(F, D) <= SAME["tc_split16"]
    # the pieces' schedule (short last pieces ordered by atomics) decides only
    # which CTA pair computes a piece: a second run is bitwise identical
    assert np.array_equal(run(wl, "tc_split16", SPARSE), F)


def test_batch_mixed_with_cutoff_and_graph_capture():
    """Gaussian instances (block-sparse) and Epanechnikov instances (cutoff)
    share one bin sort; the whole call is captured in a CUDA graph."""
    wls = [workloads.random_points(720 + k, 3000 + 997 * k, 4000.0 + 1000 * k, 10.0,
                                   300 + 70 * k, 260 + 50 * k, 25.0 + 10 * k,
                                   oracle.GAUSSIAN if k % 2 == 0 else oracle.EPANECHNIKOV)
           for k in range(5)]
    insts = []
    for wl in wls:
        pts, w = dev(wl)
        insts.append(dict(points=pts, weights=w, origin=wl.origin, cell=wl.cell, nx=wl.nx,
                          ny=wl.ny, h=wl.h, kernel=wl.kernel,
                          out=torch.empty((wl.ny, wl.nx), device="cuda")))
    outs = kde.grid_batched(insts, flags=SPARSE)
    torch.cuda.synchronize()
    first = [o.cpu().numpy() for o in outs]
    for wl, F in zip(wls, first):
        ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, wl.kernel)
        tol = TOL_SPLIT if wl.kernel == oracle.GAUSSIAN else 1e-6
        assert rel_linf(F, ref) <= tol
    for o in outs:
        o.zero_()
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            kde.grid_batched(insts, flags=kde.FLAG_SKIP_ZERO, stream=st)
    g.replay()
    torch.cuda.synchronize()
    for F, o in zip(first, outs):
        np.testing.assert_array_equal(o.cpu().numpy(), F)


def test_all_points_beyond_reach_and_empty():
    origin = workloads.FALSE_ORIGIN
    far = np.array(origin) + np.array([[-5000.0, 100.0], [100.0, 90000.0], [7e4, 7e4]])
    wl = workloads.Workload("far", far - np.array(origin), np.ones(3, np.float32), 1000.0, 10.0,
                            100, 80, 20.0, oracle.GAUSSIAN, np.array([0, 3]), 0)
    F = run(wl, "tc_split16", SPARSE)
    assert not F.any()
    empty = torch.zeros((0, 2), dtype=torch.float64, device="cuda")
    out = kde.grid(empty, None, origin, 10.0, 300, 300, 20.0, "gaussian", path="tc_split16",
                   flags=SPARSE)
    assert not out.cpu().numpy().any()


def test_one_cta_flag_conflicts():
    wl = workloads.config1()
    pts, w = dev(wl)
    with pytest.raises(RuntimeError):
        kde.grid(pts, w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, "gaussian", path="tc_split16",
                 flags=SPARSE | kde.FLAG_ONE_CTA)
