"""Degenerate inputs on every density path: no points, all-zero weights, one
point, points exactly on cell centres and cell edges, a one-row grid."""
import numpy as np
import pytest

import oracle
import workloads
from kde_testutil import TOL_FP16, TOL_FP32, TOL_SPLIT, rel_linf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2004_13653_gb300 as kde  # noqa: E402

# (path, kernel, flags, tolerance)
PATHS = [("tc_split16", "gaussian", 0, TOL_SPLIT),
         ("tc_split16", "gaussian", 8, TOL_SPLIT),      # one CTA per tile
         ("tc_split16", "gaussian", 2, TOL_SPLIT),      # block-sparse
         ("tc_fp16", "gaussian", 0, TOL_FP16),
         ("simt", "gaussian", 0, TOL_FP32),
         ("cutoff", "epanechnikov", 0, TOL_FP32),
         ("auto", "radial_quartic", 0, TOL_FP32)]
IDS = [f"{p}-{k}-{f}" for p, k, f, _ in PATHS]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kde.load(build_if_stale=True)


def run(xy, w, origin, cell, nx, ny, h, kernel, path, flags, fill=None):
    pts = torch.as_tensor(np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2),
                          device="cuda")
    wt = None if w is None else torch.as_tensor(np.asarray(w, np.float32), device="cuda")
    out = torch.full((ny, nx), 7.0 if fill is None else fill, device="cuda")
    kde.grid(pts, wt, origin, cell, nx, ny, h, kernel, out=out, path=path,
             flags=kde.FLAG_SYNC | flags)
    return out.cpu().numpy()


@pytest.mark.parametrize("path,kernel,flags,tol", PATHS, ids=IDS)
def test_no_points_writes_zeros(path, kernel, flags, tol):
    F = run(np.zeros((0, 2)), None, workloads.FALSE_ORIGIN, 10.0, 300, 260, 30.0, kernel, path,
            flags)
    assert not F.any()


@pytest.mark.parametrize("path,kernel,flags,tol", PATHS, ids=IDS)
def test_all_zero_weights(path, kernel, flags, tol):
    wl = workloads.random_points(800, 500, 2000.0, 10.0, 200, 150, 30.0, oracle.GAUSSIAN)
    F = run(wl.xy, np.zeros(wl.n), wl.origin, wl.cell, wl.nx, wl.ny, wl.h, kernel, path, flags)
    assert not F.any()


@pytest.mark.parametrize("path,kernel,flags,tol", PATHS, ids=IDS)
def test_points_on_centres_and_edges(path, kernel, flags, tol):
    """Fixes exactly at cell centres, on cell edges and on grid corners, plus
    one point alone in a far corner (its density is a lone kernel)."""
    origin = workloads.FALSE_ORIGIN
    cell, nx, ny, h = 10.0, 180, 140, 35.0
    i = np.arange(20, 160, 7)
    centres = np.stack([(i + 0.5) * cell, (i[::-1] * 0.7 + 0.5).astype(int) * cell + 5.0], 1)
    edges = np.stack([i * cell, (i * 0.5).astype(int) * cell], 1)
    corners = np.array([[0.0, 0.0], [nx * cell, 0.0], [0.0, ny * cell], [nx * cell, ny * cell]])
    lone = np.array([[3.0 * cell + 1.5, (ny - 4) * cell + 2.5]])
    local = np.concatenate([centres, edges, corners, lone])
    xy = local + np.array(origin)
    kid = oracle.KERNEL_NAMES.index(kernel) if kernel in oracle.KERNEL_NAMES else \
        oracle.RADIAL + oracle.KERNEL_NAMES.index(kernel[len("radial_"):])
    F = run(xy, None, origin, cell, nx, ny, h, kernel, path, flags)
    ref = oracle.kde_grid(xy, None, origin, cell, nx, ny, h, kid)
    # (both compact kernels here are continuous at the support's edge, where
    # points on cell edges put some pairs exactly)
    assert rel_linf(F, ref) <= tol


def test_one_row_and_one_column_grids():
    wl = workloads.random_points(801, 800, 1500.0, 10.0, 150, 1, 25.0, oracle.GAUSSIAN)
    for nx, ny in ((150, 1), (1, 150)):
        ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, nx, ny, wl.h, oracle.GAUSSIAN)
        for path, kernel, flags, tol in PATHS[:5]:
            F = run(wl.xy, wl.w, wl.origin, wl.cell, nx, ny, wl.h, kernel, path, flags)
            assert rel_linf(F, ref) <= tol, (nx, ny, path, flags)
