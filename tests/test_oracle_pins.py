"""Pins of the FP64 oracle against facts fixed outside it (CPU only).

Each test checks the oracle against something it cannot agree with by
construction: constants the paper prints (Table 1), textbook closed forms of
the kernels, invariances of the definition, an exact rational brute force, a
library routine the Gaussian case reduces to, and the differential geometry
of the Mercator projection (Eq. 1-4).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import integrate

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SAFE = {"sqrt": math.sqrt, "pi": math.pi, "__builtins__": {}}


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _k(kid):
    lib = oracle._load()
    return lambda s: lib.oracle_kernel_1d(kid, s)


# ------------------------------------------------------------ Table 1 kernels

@pytest.mark.parametrize("row", _golden_rows("table1_peaks.txt"), ids=lambda r: r[1])
def test_table1_peak_value(row):
    """f(0,0) equals the constant Table 1 prints for the kernel."""
    kid, expr = int(row[0]), row[2]
    expected = eval(expr, SAFE)
    got = oracle.kernel_1d(kid, 0.0) ** 2
    assert got == pytest.approx(expected, rel=1e-15)


@pytest.mark.parametrize("row", _golden_rows("kernel_moments.txt"), ids=lambda r: r[1])
def test_kernel_textbook_moments(row):
    """Mass, second moment and roughness match the textbook closed forms."""
    kid = int(row[0])
    mass, mu2, rough = (eval(e, SAFE) for e in row[2:5])
    k = _k(kid)
    if kid == oracle.GAUSSIAN:
        lim, pts = (-np.inf, np.inf), None
    else:
        lim, pts = (-1.0, 1.0), [0.0]
    quad = lambda f: integrate.quad(f, *lim, points=pts, epsabs=1e-13, epsrel=1e-12,
                                    limit=200)[0]
    assert quad(k) == pytest.approx(mass, rel=1e-10)
    assert quad(lambda s: s * s * k(s)) == pytest.approx(mu2, rel=1e-10)
    assert quad(lambda s: k(s) ** 2) == pytest.approx(rough, rel=1e-10)


@pytest.mark.parametrize("kid", [k for k in range(8) if k != oracle.GAUSSIAN])
def test_compact_support_inclusive(kid):
    """I(s) of Eq. 8 is 1 on |s| <= 1 and 0 outside (s in bandwidths)."""
    assert oracle.kernel_1d(kid, 1.0 + 1e-12) == 0.0
    assert oracle.kernel_1d(kid, -1.0 - 1e-12) == 0.0
    inside = oracle.kernel_1d(kid, 1.0)
    if kid == oracle.UNIFORM:
        assert inside == 0.5          # the boundary itself is inside
    else:
        assert abs(inside) < 1e-15    # the polynomial / cosine vanish there


# -------------------------------------------------------- density on a grid

@pytest.mark.parametrize("kid", range(8))
def test_grid_mass_and_normaliser(kid):
    """cell^2 * sum F = sum(w)/N when the grid covers the support.

    With h a whole number of cells and the points on cell corners the kinks of
    the compact kernels fall on cell boundaries, so the midpoint rule is exact
    for the piecewise-linear kernels and O((cell/h)^2) for the others."""
    cell, m = 1.0, 24
    h = m * cell
    nx = ny = 2 * 10 * m if kid == oracle.GAUSSIAN else 4 * m
    ox = oy = 0.0
    c = nx // 2
    xy = np.array([[c, c], [c + 3, c - 2], [c - 5, c + 1]], dtype=float)
    w = np.array([1.0, 2.5, 0.25])
    F = oracle.kde_grid(xy, w, (ox, oy), cell, nx, ny, h, kid)
    mass = cell * cell * F.sum()
    expected = w.sum() / len(w)
    tol = 1e-12 if kid in (oracle.UNIFORM, oracle.TRIANGULAR) else 2e-3
    if kid == oracle.GAUSSIAN:
        tol = 1e-9
    assert mass == pytest.approx(expected, rel=tol)
    # a wrong power of h would scale the mass by h; a weight-sum normaliser
    # instead of N would give 1 here
    assert abs(mass - 1.0) > 0.1


@pytest.mark.parametrize("kid", range(8))
def test_grid_second_moment(kid):
    """cell^2 sum (gx - x_p)^2 F = h^2 mu2 for one point (textbook mu2)."""
    rows = {int(r[0]): r for r in _golden_rows("kernel_moments.txt")}
    mu2 = eval(rows[kid][3], SAFE)
    cell, m = 1.0, 40
    h = m * cell
    nx = ny = 2 * 10 * m if kid == oracle.GAUSSIAN else 4 * m
    x0 = nx // 2
    F = oracle.kde_grid([[x0, x0]], None, (0.0, 0.0), cell, nx, ny, h, kid)
    gx = (np.arange(nx) + 0.5) * cell
    m2 = cell * cell * np.sum(F * ((gx - x0) ** 2)[None, :])
    assert m2 == pytest.approx(h * h * mu2, rel=2e-3)


def test_single_point_rank_one_and_orientation():
    """One point: F is the outer product of two 1-D profiles, peaks in the
    point's cell, and out[j, i] has j along y and i along x."""
    nx, ny, cell = 37, 23, 10.0
    xy = [[1000.0 + 12.3 * cell, 5000.0 + 7.6 * cell]]
    F = oracle.kde_grid(xy, None, (1000.0, 5000.0), cell, nx, ny, 25.0, oracle.EPANECHNIKOV)
    assert F.shape == (ny, nx)
    j, i = np.unravel_index(np.argmax(F), F.shape)
    assert (i, j) == (12, 7)
    u, s, vt = np.linalg.svd(F)
    assert s[1] < 1e-12 * s[0]


def test_reflection_symmetry():
    """Mirroring the points about the grid's vertical centre line mirrors F."""
    rng = np.random.default_rng(5)
    nx, ny, cell = 40, 30, 7.0
    ox, oy = 300.0, -200.0
    xy = np.column_stack([ox + rng.uniform(0, nx * cell, 25), oy + rng.uniform(0, ny * cell, 25)])
    w = rng.uniform(0.5, 2, 25)
    mirrored = xy.copy()
    mirrored[:, 0] = 2 * (ox + 0.5 * nx * cell) - xy[:, 0]
    for kid in (oracle.GAUSSIAN, oracle.TRICUBE, oracle.TRIANGULAR):
        F = oracle.kde_grid(xy, w, (ox, oy), cell, nx, ny, 20.0, kid)
        G = oracle.kde_grid(mirrored, w, (ox, oy), cell, nx, ny, 20.0, kid)
        np.testing.assert_allclose(G, F[:, ::-1], rtol=1e-12, atol=1e-18)


def test_transpose_and_translation():
    """Swapping x and y transposes F; shifting by whole cells shifts F."""
    rng = np.random.default_rng(6)
    n, cell = 30, 5.0
    xy = rng.uniform(40, 160, (n, 2))
    F = oracle.kde_grid(xy, None, (0, 0), cell, 40, 40, 12.0, oracle.QUARTIC)
    Ft = oracle.kde_grid(xy[:, ::-1], None, (0, 0), cell, 40, 40, 12.0, oracle.QUARTIC)
    np.testing.assert_allclose(Ft, F.T, rtol=1e-12, atol=1e-18)
    Fs = oracle.kde_grid(xy + [3 * cell, -2 * cell], None, (0, 0), cell, 40, 40, 12.0,
                         oracle.QUARTIC)
    np.testing.assert_allclose(Fs[5:35, 8:38], F[7:37, 5:35], rtol=1e-11, atol=1e-18)


def test_permutation_invariance():
    rng = np.random.default_rng(7)
    xy = rng.uniform(0, 100, (50, 2))
    w = rng.uniform(0.5, 2, 50)
    perm = rng.permutation(50)
    F = oracle.kde_grid(xy, w, (0, 0), 5.0, 20, 20, 15.0, oracle.GAUSSIAN)
    G = oracle.kde_grid(xy[perm], w[perm], (0, 0), 5.0, 20, 20, 15.0, oracle.GAUSSIAN)
    np.testing.assert_allclose(G, F, rtol=1e-13)


def _exact_k(kid, s: Fraction) -> Fraction:
    a = abs(s)
    if a > 1:
        return Fraction(0)
    if kid == oracle.UNIFORM:
        return Fraction(1, 2)
    if kid == oracle.TRIANGULAR:
        return 1 - a
    if kid == oracle.EPANECHNIKOV:
        return Fraction(3, 4) * (1 - s * s)
    if kid == oracle.QUARTIC:
        return Fraction(15, 16) * (1 - s * s) ** 2
    if kid == oracle.TRIWEIGHT:
        return Fraction(35, 32) * (1 - s * s) ** 3
    if kid == oracle.TRICUBE:
        return Fraction(70, 81) * (1 - a ** 3) ** 3
    raise ValueError(kid)


@pytest.mark.parametrize("kid", [0, 1, 2, 3, 4, 5])
def test_exact_rational_brute_force(kid):
    """Tiny inputs summed in exact rational arithmetic (n <= 5, 4x3 grid)."""
    rng = np.random.default_rng(100 + kid)
    n, nx, ny = 5, 4, 3
    cell, h = Fraction(5, 2), Fraction(7, 2)
    ox, oy = Fraction(-3, 4), Fraction(1, 8)
    pts = [(Fraction(int(rng.integers(-8, 90)), 8), Fraction(int(rng.integers(-8, 70)), 8))
           for _ in range(n)]
    ws = [Fraction(int(rng.integers(1, 9)), 4) for _ in range(n)]
    exact = np.empty((ny, nx))
    for j in range(ny):
        for i in range(nx):
            gx = ox + (i + Fraction(1, 2)) * cell
            gy = oy + (j + Fraction(1, 2)) * cell
            acc = sum(wp * _exact_k(kid, (gx - x) / h) * _exact_k(kid, (gy - y) / h)
                      for (x, y), wp in zip(pts, ws))
            exact[j, i] = float(acc / (n * h * h))
    got = oracle.kde_grid([[float(x), float(y)] for x, y in pts], [float(v) for v in ws],
                          (float(ox), float(oy)), float(cell), nx, ny, float(h), kid)
    assert np.count_nonzero(exact) > 3
    np.testing.assert_allclose(got, exact, rtol=1e-13, atol=1e-16)


def test_gaussian_is_a_matrix_product():
    """For the Gaussian, F = c A B^T with A, B the 1-D profiles (numpy matmul)."""
    rng = np.random.default_rng(8)
    n, nx, ny, cell, h = 40, 17, 13, 9.0, 14.0
    xy = rng.uniform(-20, 170, (n, 2))
    w = rng.uniform(0.5, 2, n)
    gx = (np.arange(nx) + 0.5) * cell
    gy = (np.arange(ny) + 0.5) * cell
    A = np.exp(-0.5 * ((gx[:, None] - xy[None, :, 0]) / h) ** 2)
    B = w[None, :] * np.exp(-0.5 * ((gy[:, None] - xy[None, :, 1]) / h) ** 2)
    expected = (B @ A.T) / (2 * np.pi * n * h * h)
    got = oracle.kde_grid(xy, w, (0, 0), cell, nx, ny, h, oracle.GAUSSIAN)
    np.testing.assert_allclose(got, expected, rtol=1e-12)


def test_sampled_cells_match_full_grid():
    rng = np.random.default_rng(9)
    xy = rng.uniform(0, 300, (60, 2))
    F = oracle.kde_grid(xy, None, (0, 0), 10.0, 30, 30, 25.0, oracle.COSINE)
    cells = rng.choice(900, 50, replace=False)
    got = oracle.kde_cells(xy, None, (0, 0), 10.0, 30, 30, 25.0, oracle.COSINE, cells)
    np.testing.assert_array_equal(got, F.reshape(-1)[cells])


def test_empty_input_is_zero():
    out = oracle.kde_cells(np.zeros((0, 2)), None, (0, 0), 1.0, 3, 3, 1.0, oracle.GAUSSIAN)
    assert out.shape == (3, 3) and not out.any()


# ---------------------------------------------------------------- Mercator

def test_mercator_equator_and_meridian():
    xy = oracle.mercator([[0.0, 0.0], [10.0, 0.0], [0.0, 45.0]], 0.0)
    # q(0) = ln tan(pi/4) = 0 up to the rounding of tan(pi/4) in FP64
    assert xy[0, 0] == 0.0 and abs(xy[0, 1]) < 1e-8
    assert abs(xy[1, 1]) < 1e-8
    assert xy[1, 0] == pytest.approx(oracle.WGS84_A * math.radians(10.0), rel=1e-15)
    assert xy[2, 0] == 0.0 and xy[2, 1] > 0


@pytest.mark.parametrize("lat0", [0.0, 31.35, 37.45, 60.0])
def test_mercator_parallel_radius_from_reduced_latitude(lat0):
    """r0 = a cos(beta) with the reduced latitude tan(beta) = sqrt(1-e^2) tan(phi0):
    the distance of the standard parallel from the polar axis."""
    beta = math.atan(math.sqrt(1 - oracle.WGS84_E2) * math.tan(math.radians(lat0)))
    r0 = oracle.WGS84_A * math.cos(beta)
    xy = oracle.mercator([[1.0, 0.0]], lat0)
    assert xy[0, 0] / math.radians(1.0) == pytest.approx(r0, rel=1e-13)


@pytest.mark.parametrize("lat", [-60.0, -10.0, 0.5, 31.35, 37.45, 75.0])
def test_mercator_isometric_latitude_derivative(lat):
    """dq/dphi = (1 - e^2) / ((1 - e^2 sin^2 phi) cos phi): the textbook
    derivative of the isometric latitude, against central differences."""
    e2 = oracle.WGS84_E2
    lat0 = 0.0  # r0 = a
    d = 1e-4
    ya = oracle.mercator([[0.0, lat - d]], lat0)[0, 1]
    yb = oracle.mercator([[0.0, lat + d]], lat0)[0, 1]
    dq = (yb - ya) / oracle.WGS84_A / math.radians(2 * d)
    phi = math.radians(lat)
    expected = (1 - e2) / ((1 - e2 * math.sin(phi) ** 2) * math.cos(phi))
    assert dq == pytest.approx(expected, rel=1e-7)


def test_mercator_inverse_round_trip():
    """Inverting y by the fixed-point iteration for the ellipsoidal isometric
    latitude recovers the latitude to ~1e-12 degrees."""
    e = math.sqrt(oracle.WGS84_E2)
    lats = np.linspace(-70, 70, 29)
    ll = np.column_stack([np.full_like(lats, 121.68), lats])
    xy = oracle.mercator(ll, 0.0)
    for (lon, lat), (x, y) in zip(ll, xy):
        q = y / oracle.WGS84_A
        phi = 2 * math.atan(math.exp(q)) - math.pi / 2
        for _ in range(60):
            s = e * math.sin(phi)
            phi = 2 * math.atan(math.exp(q) * ((1 + s) / (1 - s)) ** (e / 2)) - math.pi / 2
        assert math.degrees(phi) == pytest.approx(lat, abs=1e-11)
        assert math.degrees(x / oracle.WGS84_A) == pytest.approx(lon, rel=1e-14)


# ------------------------------------------------------- Douglas-Peucker

def test_ved_closed_forms():
    assert oracle.ved((3, 4), (0, 0), (10, 0)) == pytest.approx(4.0)
    assert oracle.ved((3, -4), (0, 0), (10, 0)) == pytest.approx(4.0)
    assert oracle.ved((20, 4), (0, 0), (10, 0)) == pytest.approx(4.0)  # line, not segment
    assert oracle.ved((3, 4), (1, 1), (1, 1)) == pytest.approx(math.hypot(2, 3))
    assert oracle.ved((1, 1), (0, 0), (2, 2)) == pytest.approx(0.0, abs=1e-15)


def _dp_textbook(pts, eps):
    """Recursive textbook Douglas-Peucker on a tiny polyline."""
    keep = [False] * len(pts)
    keep[0] = keep[-1] = True

    def rec(s, e):
        best, kbest = -1.0, -1
        for k in range(s + 1, e):
            d = oracle.ved(pts[k], pts[s], pts[e])
            if d > best:
                best, kbest = d, k
        if kbest >= 0 and best > eps:
            keep[kbest] = True
            rec(s, kbest)
            rec(kbest, e)

    rec(0, len(pts) - 1)
    return np.array(keep)


def test_dp_matches_recursion_and_property():
    rng = np.random.default_rng(11)
    for trial in range(30):
        n = int(rng.integers(2, 40))
        pts = np.cumsum(rng.normal(0, 10, (n, 2)), axis=0)
        eps = float(rng.uniform(0, 15))
        keep = oracle.douglas_peucker(pts, [0, n], eps)
        np.testing.assert_array_equal(keep, _dp_textbook(pts, eps))
        kept = np.nonzero(keep)[0]
        for a, b in zip(kept[:-1], kept[1:]):
            for k in range(a + 1, b):
                assert oracle.ved(pts[k], pts[a], pts[b]) <= eps


def test_dp_zero_threshold_keeps_everything():
    """At eps = 0 nothing is removed (compression ratio 0, Table 4 first row)
    when no three consecutive fixes are exactly collinear."""
    rng = np.random.default_rng(12)
    pts = rng.normal(0, 100, (500, 2))
    off = [0, 100, 250, 500]
    keep = oracle.douglas_peucker(pts, off, 0.0)
    assert keep.all()


def test_dp_trajectories_are_independent():
    rng = np.random.default_rng(13)
    a = np.cumsum(rng.normal(0, 5, (50, 2)), axis=0)
    b = np.cumsum(rng.normal(0, 5, (30, 2)), axis=0)
    both = oracle.douglas_peucker(np.vstack([a, b]), [0, 50, 80], 4.0)
    np.testing.assert_array_equal(both[:50], oracle.douglas_peucker(a, [0, 50], 4.0))
    np.testing.assert_array_equal(both[50:], oracle.douglas_peucker(b, [0, 30], 4.0))
