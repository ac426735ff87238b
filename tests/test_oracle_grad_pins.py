"""Pins of the oracle's analytic gradients and LSCV loss (CPU only).

The analytic vector-Jacobian product and the LSCV gradient are checked against
central finite differences of the (separately pinned) FP64 forward, and the
LSCV's integral term against the exact Gaussian closed form
int f^2 = sum_pq w_p w_q exp(-|x_p-x_q|^2 / 4h^2) / (4 pi N^2 h^2).
"""
import math

import numpy as np
import pytest

import oracle


def _case(seed=21, n=6):
    rng = np.random.default_rng(seed)
    nx, ny, cell = 24, 18, 10.0
    origin = (1000.0, -500.0)
    xy = np.column_stack([origin[0] + rng.uniform(40, 200, n), origin[1] + rng.uniform(40, 140, n)])
    w = rng.uniform(0.5, 2.0, n)
    G = rng.normal(0, 1, (ny, nx))
    return xy, w, origin, cell, nx, ny, 17.0, G


def _L(xy, w, origin, cell, nx, ny, h, G):
    F = oracle.kde_grid(xy, w, origin, cell, nx, ny, h, oracle.GAUSSIAN)
    return float(np.sum(G * F))


def test_vjp_matches_central_differences():
    xy, w, origin, cell, nx, ny, h, G = _case()
    gw, gxy, gh = oracle.kde_vjp_gauss(xy, w, origin, cell, nx, ny, h, G)
    L = lambda **kw: _L(kw.get("xy", xy), kw.get("w", w), origin, cell, nx, ny,
                       kw.get("h", h), G)
    eps = 1e-3
    for p in range(len(w)):
        wp, wm = w.copy(), w.copy()
        wp[p] += eps
        wm[p] -= eps
        assert gw[p] == pytest.approx((L(w=wp) - L(w=wm)) / (2 * eps), rel=1e-6, abs=1e-12)
        for c in (0, 1):
            a, b = xy.copy(), xy.copy()
            a[p, c] += eps
            b[p, c] -= eps
            fd = (L(xy=a) - L(xy=b)) / (2 * eps)
            assert gxy[p, c] == pytest.approx(fd, rel=1e-5, abs=1e-12)
    fd_h = (L(h=h + eps) - L(h=h - eps)) / (2 * eps)
    assert gh == pytest.approx(fd_h, rel=1e-6)


def test_vjp_subset_matches_full():
    xy, w, origin, cell, nx, ny, h, G = _case(22, 9)
    gw, gxy, _ = oracle.kde_vjp_gauss(xy, w, origin, cell, nx, ny, h, G)
    sel = [7, 2, 4]
    sw, sxy, sh = oracle.kde_vjp_gauss(xy, w, origin, cell, nx, ny, h, G, pts=sel)
    assert sh is None
    np.testing.assert_allclose(sw, gw[sel], rtol=1e-14)
    np.testing.assert_allclose(sxy, gxy[sel], rtol=1e-14)


def test_single_point_gradient_closed_form():
    """One point, G = one-hot at cell (i,j): dF_ij/dx_p = F_ij (gx_i - x_p)/h^2."""
    nx, ny, cell, h = 9, 7, 10.0, 13.0
    xy = np.array([[41.0, 33.0]])
    G = np.zeros((ny, nx))
    i, j = 5, 2
    G[j, i] = 1.0
    F = oracle.kde_grid(xy, [1.5], (0, 0), cell, nx, ny, h, oracle.GAUSSIAN)
    gw, gxy, gh = oracle.kde_vjp_gauss(xy, [1.5], (0, 0), cell, nx, ny, h, G)
    gx, gy = (i + 0.5) * cell, (j + 0.5) * cell
    assert gxy[0, 0] == pytest.approx(F[j, i] * (gx - xy[0, 0]) / h ** 2, rel=1e-12)
    assert gxy[0, 1] == pytest.approx(F[j, i] * (gy - xy[0, 1]) / h ** 2, rel=1e-12)
    assert gw[0] == pytest.approx(F[j, i] / 1.5, rel=1e-12)
    r2 = (gx - xy[0, 0]) ** 2 + (gy - xy[0, 1]) ** 2
    assert gh == pytest.approx(F[j, i] * (r2 / h ** 3 - 2 / h), rel=1e-12)


def test_lscv_gradient_matches_central_differences():
    xy, w, origin, cell, nx, ny, h, _ = _case(23, 7)

    def loss(xy_, w_, h_):
        F = oracle.kde_grid(xy_, w_, origin, cell, nx, ny, h_, oracle.GAUSSIAN)
        return oracle.lscv_loss(F, xy_, w_, origin, cell, nx, ny, h_)

    L, gw, gxy, gh = oracle.lscv_value_and_grad(xy, w, origin, cell, nx, ny, h)
    assert L == pytest.approx(loss(xy, w, h), rel=1e-14)
    eps = 1e-3
    for p in range(len(w)):
        wp, wm = w.copy(), w.copy()
        wp[p] += eps
        wm[p] -= eps
        assert gw[p] == pytest.approx((loss(xy, wp, h) - loss(xy, wm, h)) / (2 * eps),
                                      rel=1e-5, abs=1e-13)
        for c in (0, 1):
            a, b = xy.copy(), xy.copy()
            a[p, c] += eps
            b[p, c] -= eps
            fd = (loss(a, w, h) - loss(b, w, h)) / (2 * eps)
            assert gxy[p, c] == pytest.approx(fd, rel=1e-4, abs=1e-13)
    fd_h = (loss(xy, w, h + eps) - loss(xy, w, h - eps)) / (2 * eps)
    assert gh == pytest.approx(fd_h, rel=1e-5)


def test_lscv_square_term_matches_gaussian_closed_form():
    """cell^2 sum F^2 -> int f^2 (exact for the Gaussian) on a fine grid."""
    rng = np.random.default_rng(24)
    n, h, cell = 5, 20.0, 2.0
    nx = ny = 200
    xy = rng.uniform(150, 250, (n, 2))
    w = rng.uniform(0.5, 2, n)
    F = oracle.kde_grid(xy, w, (0, 0), cell, nx, ny, h, oracle.GAUSSIAN)
    grid_term = cell * cell * np.sum(F * F)
    d2 = ((xy[:, None, :] - xy[None, :, :]) ** 2).sum(-1)
    exact = np.sum(w[:, None] * w[None, :] * np.exp(-d2 / (4 * h * h))) / (
        4 * math.pi * n * n * h * h)
    assert grid_term == pytest.approx(exact, rel=1e-6)
