"""Douglas-Peucker on the GPU (Sec. III-B, Eq. 9, the level-synchronous form
of Sec. IV-A) against the oracle's sequential recursion: the keep masks must be
identical bit for bit (the VED decides an index, and both sides evaluate it in
FP64 with the same rounding), the compacted points and offsets must match."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2004_13653_gb300 as kde  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kde.load(build_if_stale=True)


def check(xy, offsets, eps):
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
    n = xy.shape[0]
    pts = torch.as_tensor(xy, device="cuda")
    off = None if offsets is None else torch.as_tensor(np.asarray(offsets, np.int64),
                                                       device="cuda")
    keep, out, out_off, its = kde.dp_simplify(pts, off, eps)
    torch.cuda.synchronize()
    host_off = np.array([0, n], np.int64) if offsets is None else np.asarray(offsets, np.int64)
    ref = oracle.douglas_peucker(xy, host_off, eps).astype(np.uint8)
    k = keep.cpu().numpy()
    np.testing.assert_array_equal(k, ref)
    np.testing.assert_array_equal(out.cpu().numpy(), xy[ref.astype(bool)])
    cum = np.concatenate([[0], np.cumsum(ref)])
    np.testing.assert_array_equal(out_off.cpu().numpy(), cum[host_off])
    return k, its


def test_lane_trajectories_2M_eps10():
    """The 2M raw lane fixes (4000 vessels x 500) at eps = 10 m, the
    thinning step upstream of the bandwidth fit."""
    wl = workloads.config5_raw()
    k, its = check(wl.xy, wl.offsets, 10.0)
    assert 0.02 < k.mean() < 0.9 and its > 3


@pytest.mark.parametrize("eps", [0.0, 1.0, 50.0, 5000.0])
def test_thresholds_config2(eps):
    wl = workloads.config2()
    k, _ = check(wl.xy, wl.offsets, eps)
    if eps == 5000.0:   # lanes of a 50 km box: few points survive
        assert k.mean() < 0.05


def test_small_and_degenerate_trajectories():
    """Lengths 0 (empty), 1, 2, 3; duplicated points (zero-length segments:
    the VED is then the distance to the start); collinear runs (all VEDs 0);
    an exact tie between two points (the first one is kept)."""
    rng = np.random.default_rng(11)
    parts, lens = [], []
    parts.append(np.zeros((0, 2))); lens.append(0)
    parts.append(rng.normal(size=(1, 2))); lens.append(1)
    parts.append(rng.normal(size=(2, 2))); lens.append(2)
    parts.append(rng.normal(size=(3, 2))); lens.append(3)
    loop = rng.normal(size=(6, 2)) * 10
    parts.append(np.vstack([loop, loop[:1]])); lens.append(7)       # closed: ends coincide
    parts.append(np.repeat(rng.normal(size=(4, 2)), 3, axis=0)); lens.append(12)
    parts.append(np.stack([np.linspace(0, 100, 50), np.linspace(5, 55, 50)], 1)); lens.append(50)
    parts.append(np.array([[0.0, 0.0], [1.0, 1.0], [2.0, -1.0], [3.0, 0.0]])); lens.append(4)
    parts.append(np.array([[0.0, 0.0], [1.0, 2.0], [2.0, 2.0], [3.0, 0.0]])); lens.append(4)
    xy = np.vstack(parts) + np.array(workloads.FALSE_ORIGIN)
    offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    for eps in (0.0, 0.5, 1.0, 3.0):
        check(xy, offsets, eps)


def test_single_trajectory_without_offsets():
    """One long random walk (deep recursion), offsets NULL."""
    rng = np.random.default_rng(12)
    xy = np.cumsum(rng.normal(size=(200_000, 2)) * 30.0, axis=0) + 1e6
    k, its = check(xy, None, 25.0)
    assert its > 10


def test_empty_input():
    pts = torch.zeros((0, 2), dtype=torch.float64, device="cuda")
    keep, out, out_off, its = kde.dp_simplify(pts, None, 1.0)
    assert keep.numel() == 0 and out.shape[0] == 0 and out_off.cpu().tolist() == [0, 0]


def test_invalid_arguments():
    pts = torch.zeros((10, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):
        kde.dp_simplify(pts, None, -1.0)
    bad = torch.tensor([0, 4, 9], dtype=torch.int64, device="cuda")   # does not end at n
    with pytest.raises(RuntimeError):
        kde.dp_simplify(pts, bad, 1.0)
    pts[3, 1] = float("nan")
    with pytest.raises(RuntimeError):
        kde.dp_simplify(pts, None, 1.0)
