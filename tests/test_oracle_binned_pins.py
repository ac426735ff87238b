"""Pins of the oracle's binned estimator (Sec. IV-B, Algorithm 3, Eq. 7)
(CPU only): hand-computed interpolation, brute-force counts, the stencil of
a single count, and closeness to the direct sum when the bins are fine."""
import numpy as np
import pytest

import oracle


def test_interpolation_hand_example():
    """Fixes in cells (1,1) and (4,2): c_max = 3, interpolated cells
    round(1 + c, 1 + c/3) = (2,1) and (3,2)."""
    xy = np.array([[1.5, 1.5], [4.5, 2.5]])
    counts, added = oracle.count_matrix(xy, [0, 2], (0.0, 0.0), 1.0, 6, 4)
    assert added == 2
    expect = np.zeros((4, 6), np.int32)
    for i, j in [(1, 1), (4, 2), (2, 1), (3, 2)]:
        expect[j, i] += 1
    np.testing.assert_array_equal(counts, expect)
    no_interp, added0 = oracle.count_matrix(xy, [0, 2], (0.0, 0.0), 1.0, 6, 4, False)
    assert added0 == 0 and no_interp.sum() == 2


def test_no_interpolation_across_trajectories_or_adjacent_cells():
    xy = np.array([[0.5, 0.5], [1.5, 1.5], [5.5, 3.5], [0.2, 3.9]])
    counts, added = oracle.count_matrix(xy, [0, 2, 4], (0.0, 0.0), 1.0, 6, 4)
    # (0,0)->(1,1): c_max = 1, nothing added; the jump (1,1)->(5,3) is between trajectories
    # (5,3)->(0,3): c_max = 5, four cells added in row 3
    assert added == 4
    assert counts[3].tolist() == [1, 1, 1, 1, 1, 1]


def test_counts_match_brute_force():
    rng = np.random.default_rng(31)
    xy = rng.uniform(-5, 65, (400, 2))
    counts, _ = oracle.count_matrix(xy, [0, 400], (0.0, 0.0), 2.5, 24, 24, interpolate=False)
    ref = np.zeros((24, 24), np.int32)
    for x, y in xy:
        i, j = int(np.floor(x / 2.5)), int(np.floor(y / 2.5))
        if 0 <= i < 24 and 0 <= j < 24:
            ref[j, i] += 1
    np.testing.assert_array_equal(counts, ref)


@pytest.mark.parametrize("kid", [oracle.EPANECHNIKOV, oracle.GAUSSIAN, oracle.TRIANGULAR])
def test_single_count_gives_the_stencil(kid):
    counts = np.zeros((15, 15), np.int32)
    counts[7, 7] = 1
    out = oracle.convolve(counts, 10.0, 30.0, kid, 7, 3)
    s = np.arange(-3, 4) * 10.0 / 30.0
    k = oracle.kernel_1d(kid, s)
    expect = np.zeros((15, 15))
    expect[4:11, 4:11] = np.outer(k, k) / (3 * 30.0 ** 2)
    np.testing.assert_allclose(out, expect, rtol=1e-14, atol=1e-20)


def test_fine_bins_approach_the_direct_sum():
    """Without interpolation and with cells much smaller than h, the binned
    estimator is the direct sum with points moved to cell centres: error
    O(cell/h) relative."""
    rng = np.random.default_rng(32)
    n, nx, cell, h = 300, 80, 1.0, 12.0
    xy = rng.uniform(20, 60, (n, 2))
    counts, _ = oracle.count_matrix(xy, [0, n], (0.0, 0.0), cell, nx, nx, interpolate=False)
    window = 2 * int(h / cell) + 1
    binned = oracle.convolve(counts, cell, h, oracle.EPANECHNIKOV, window, n)
    direct = oracle.kde_grid(xy, None, (0.0, 0.0), cell, nx, nx, h, oracle.EPANECHNIKOV)
    err = np.max(np.abs(binned - direct)) / np.max(direct)
    assert err < 2 * cell / h
