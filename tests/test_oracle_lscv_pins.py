"""Pins of the oracle's grid LSCV loss (CPU only).

The loss is the grid form of least-squares cross-validation (the paper picks
the bandwidth by eye, Sec. V-D; this quantitative form is the library's own
reading):

    L = cell^2 sum_ij F_ij^2 - (2/N) sum_p w_p bilerp(F - F_p, x_p),

F_p being point p's own term on the grid.  Each pin below fixes a part of it
from outside the oracle's LSCV code: the leave-one-out bracket by recomputing
the grid without the point and interpolating it with scipy; the bilinear taps
by a linear field they must reproduce; the zero extension by points outside
the grid; a single point by the definition (nothing is left out of it); and
the whole loss by its convergence to the exact Gaussian LSCV as the cell
shrinks.
"""
import math

import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator

import oracle


def _bilerp_zero_outside(F, origin, cell, x, y):
    """Bilinear interpolation of F (values at cell centres) at (x, y), with
    zero beyond the grid: F padded by a ring of zeros, 0 farther out."""
    ny, nx = F.shape
    P = np.zeros((ny + 2, nx + 2))
    P[1:-1, 1:-1] = F
    gx = origin[0] + (np.arange(-1, nx + 1) + 0.5) * cell
    gy = origin[1] + (np.arange(-1, ny + 1) + 0.5) * cell
    f = RegularGridInterpolator((gy, gx), P, method="linear", bounds_error=False, fill_value=0.0)
    return float(f([[y, x]])[0])


def _case(seed):
    rng = np.random.default_rng(seed)
    nx, ny, cell, h = 20, 16, 10.0, 15.0
    origin = (500.0, -300.0)
    xy = np.column_stack([origin[0] + rng.uniform(20, 180, 7), origin[1] + rng.uniform(20, 140, 7)])
    # one point just inside the last cell centre row, one beyond the grid's edge
    # by less than half a cell (partial taps), one far outside (no taps)
    xy = np.vstack([xy, [origin[0] + 197.0, origin[1] + 80.0], [origin[0] + 203.0, origin[1] + 5.0],
                    [origin[0] - 60.0, origin[1] + 50.0]])
    w = rng.uniform(0.5, 2.0, len(xy))
    return xy, w, origin, cell, nx, ny, h


def test_leave_one_out_bracket_is_the_interpolated_density_of_the_other_points():
    xy, w, origin, cell, nx, ny, h = _case(31)
    n = len(w)
    F = oracle.kde_grid(xy, w, origin, cell, nx, ny, h, oracle.GAUSSIAN)
    loo = 0.0
    for p in range(n):
        keep = np.arange(n) != p
        # the grid of the other points with the full sample's 1/(N h^2)
        Fm = oracle.kde_grid(xy[keep], w[keep], origin, cell, nx, ny, h,
                             oracle.GAUSSIAN) * (n - 1) / n
        loo += w[p] * _bilerp_zero_outside(Fm, origin, cell, xy[p, 0], xy[p, 1])
    brute = cell * cell * np.sum(F * F) - 2.0 / n * loo
    assert oracle.lscv_loss(F, xy, w, origin, cell, nx, ny, h) == pytest.approx(brute, rel=1e-12)


@pytest.mark.parametrize("where", [(105.0, 55.0), (113.7, 41.2), (1.0, 158.5)],
                         ids=["cell centre", "off centre", "corner"])
def test_single_point_has_no_leave_one_out_term(where):
    origin, cell, nx, ny, h = (0.0, 0.0), 10.0, 20, 16, 12.0
    xy = np.array([where])
    F = oracle.kde_grid(xy, [1.7], origin, cell, nx, ny, h, oracle.GAUSSIAN)
    L = oracle.lscv_loss(F, xy, [1.7], origin, cell, nx, ny, h)
    assert L == pytest.approx(cell * cell * np.sum(F * F), rel=1e-13)


def test_bilinear_taps_reproduce_a_linear_field():
    # h far below the cell: every point's own term at its four cell centres
    # underflows to zero, leaving cell^2 sum F^2 - (2/N) sum_p w_p F(x_p)
    origin, cell, nx, ny, h = (-40.0, 70.0), 8.0, 13, 9, 8e-3
    gx = origin[0] + (np.arange(nx) + 0.5) * cell
    gy = origin[1] + (np.arange(ny) + 0.5) * cell
    lin = lambda x, y: 3.0 + 0.25 * (x - origin[0]) - 0.7 * (y - origin[1])
    F = lin(gx[None, :], gy[:, None])
    rng = np.random.default_rng(32)
    # strictly between cell centres, at least a tenth of a cell from each
    fi = rng.integers(0, nx - 1, 12) + rng.uniform(0.1, 0.9, 12)
    fj = rng.integers(0, ny - 1, 12) + rng.uniform(0.1, 0.9, 12)
    xy = np.column_stack([origin[0] + (fi + 0.5) * cell, origin[1] + (fj + 0.5) * cell])
    w = rng.uniform(0.5, 2.0, 12)
    expect = cell * cell * np.sum(F * F) - 2.0 / 12 * np.sum(w * lin(xy[:, 0], xy[:, 1]))
    assert oracle.lscv_loss(F, xy, w, origin, cell, nx, ny, h) == pytest.approx(expect, rel=1e-12)


def test_points_beyond_the_grid_read_zeros():
    origin, cell, nx, ny, h = (0.0, 0.0), 10.0, 6, 5, 1e-2
    F = np.random.default_rng(33).uniform(1.0, 2.0, (ny, nx))
    sq = cell * cell * np.sum(F * F)
    # a point more than half a cell beyond the grid has no taps
    L = oracle.lscv_loss(F, np.array([[-6.0, 20.0]]), [1.0], origin, cell, nx, ny, h)
    assert L == pytest.approx(sq, rel=1e-14)
    # a quarter cell left of the first column's centres, on row 2's centre:
    # cell (0, 2) holds 3/4 of the weight, the zero ring beyond the edge 1/4
    L = oracle.lscv_loss(F, np.array([[2.5, 25.0]]), [1.0], origin, cell, nx, ny, h)
    assert L == pytest.approx(sq - 2.0 * 0.75 * F[2, 0], rel=1e-14)


def test_grid_loss_converges_to_the_exact_gaussian_lscv():
    """With the Gaussian, int f^2 and the leave-one-out densities have closed
    forms; the grid loss approaches that exact LSCV as the cell shrinks."""
    rng = np.random.default_rng(5)
    n, h = 5, 20.0
    xy = rng.uniform(150, 250, (n, 2))
    w = rng.uniform(0.5, 2.0, n)
    d2 = ((xy[:, None, :] - xy[None, :, :]) ** 2).sum(-1)
    sq = np.sum(w[:, None] * w[None, :] * np.exp(-d2 / (4 * h * h))) / (4 * math.pi * n * n * h * h)
    K = np.exp(-d2 / (2 * h * h)) / (2 * math.pi * n * h * h)
    np.fill_diagonal(K, 0.0)
    exact = sq - 2.0 / n * np.sum(w * (K @ w))
    errs = []
    for cell in (h / 4, h / 8, h / 16):
        m = int(round(400 / cell))
        F = oracle.kde_grid(xy, w, (0.0, 0.0), cell, m, m, h, oracle.GAUSSIAN)
        errs.append(abs(oracle.lscv_loss(F, xy, w, (0.0, 0.0), cell, m, m, h) - exact) / abs(exact))
    assert errs[0] > 3 * errs[1] > 9 * errs[2]
    assert errs[2] < 5e-4
