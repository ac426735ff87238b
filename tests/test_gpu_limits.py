"""Size limits: the largest grid the ABI accepts (nx * ny just below 2^31
cells) and a point count in the hundreds of millions, on the tensor-core,
cutoff and SIMT paths, checked against the FP64 oracle on sampled cells."""
import numpy as np
import pytest

import oracle
import workloads
from kde_testutil import TOL_FP32, TOL_SPLIT, rel_linf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2004_13653_gb300 as kde  # noqa: E402

SIDE = 46340  # 46340^2 = 2,147,395,600 < 2^31


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kde.load(build_if_stale=True)


def sampled(out, cells):
    idx = torch.as_tensor(cells, device=out.device)
    return out.reshape(-1)[idx].cpu().numpy()


def corner_and_random_cells(nx, ny, extra, seed):
    rng = np.random.default_rng(seed)
    fixed = [0, nx - 1, (ny - 1) * nx, ny * nx - 1]
    return np.unique(np.concatenate([fixed, extra, rng.integers(0, nx * ny, 64)]))


@pytest.mark.parametrize("path,kid,tol", [("tc_split16", oracle.GAUSSIAN, TOL_SPLIT),
                                          ("cutoff", oracle.EPANECHNIKOV, TOL_FP32)])
def test_largest_grid(path, kid, tol):
    """46340 x 46340 cells of 10 m; 300 points spread over the grid and a
    cluster in the last tile row/column (ragged edge of the largest grid)."""
    rng = np.random.default_rng(900)
    box = SIDE * 10.0
    local = np.concatenate([rng.uniform(0, box, (200, 2)),
                            box - rng.uniform(0, 300.0, (100, 2))])
    w = rng.uniform(0.5, 2.0, local.shape[0]).astype(np.float32)
    origin = workloads.FALSE_ORIGIN
    xy = local + np.array(origin)
    pts = torch.as_tensor(xy, device="cuda")
    out = kde.grid(pts, torch.as_tensor(w, device="cuda"), origin, 10.0, SIDE, SIDE, 40.0, kid,
                   path=path, flags=kde.FLAG_SYNC)
    # cells next to points (non-zero density) plus corners and random cells
    near = np.floor(local[:40] / 10.0).astype(np.int64)
    cells = corner_and_random_cells(SIDE, SIDE, near[:, 1] * SIDE + near[:, 0], 901)
    ref = oracle.kde_cells(xy, w, origin, 10.0, SIDE, SIDE, 40.0, kid, cells)
    got = sampled(out, cells)
    assert np.max(ref) > 0
    assert rel_linf(got, ref) <= tol
    del out
    torch.cuda.empty_cache()


@pytest.mark.parametrize("path,tol", [("tc_split16", TOL_SPLIT), ("simt", TOL_FP32)])
def test_many_points_small_grid(path, tol):
    """2^27 = 134M points (generated on the device) on a 48 x 40 grid."""
    n = 1 << 27
    g = torch.Generator(device="cuda").manual_seed(902)
    origin = workloads.FALSE_ORIGIN
    local = torch.rand((n, 2), generator=g, device="cuda", dtype=torch.float64) * 500.0 - 10.0
    pts = local + torch.tensor(origin, dtype=torch.float64, device="cuda")
    del local
    out = kde.grid(pts, None, origin, 10.0, 48, 40, 15.0, "gaussian", path=path,
                   flags=kde.FLAG_SYNC)
    cells = np.array([0, 47, 20 * 48 + 24, 39 * 48 + 47])
    got = sampled(out, cells)
    ref = oracle.kde_cells(pts.cpu().numpy(), None, origin, 10.0, 48, 40, 15.0,
                           oracle.GAUSSIAN, cells)
    assert rel_linf(got, ref) <= tol
    del pts, out
    torch.cuda.empty_cache()
