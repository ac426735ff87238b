"""Pins of the oracle's radial kernels (kernel ids 8..15: Table 1 profiles
on the unit disk, K(u) = c k(|u|)), against facts fixed outside the oracle:
  - each K integrates to one over the plane (adaptive quadrature of
    2 pi r K(r), scipy) -- a wrong normalising constant fails;
  - the density of one point is a function of the distance alone (rotating
    the offset leaves F unchanged) and vanishes outside the disk, where the
    product kernel of Table 1 does not (the corner of the square support);
  - the radial Gaussian is the product Gaussian (exp(-r^2/2) factorises).
"""
import math

import numpy as np
import pytest

import oracle

scipy_integrate = pytest.importorskip("scipy.integrate")

COMPACT = [k for k in range(8) if k != oracle.GAUSSIAN]


@pytest.mark.parametrize("kid", range(8), ids=oracle.KERNEL_NAMES)
def test_radial_kernel_integrates_to_one(kid):
    upper = 12.0 if kid == oracle.GAUSSIAN else 1.0
    val, err = scipy_integrate.quad(lambda r: 2 * math.pi * r * oracle.kernel_radial(kid, r),
                                    0.0, upper, epsabs=1e-13, epsrel=1e-13, limit=200)
    assert abs(val - 1.0) < 1e-10


def _single_point_density(kid, offsets, h=1.0):
    """F at cells whose centres sit at the given offsets (in h) from one
    point: a grid of one cell per offset, the point placed accordingly."""
    out = []
    for dx, dy in offsets:
        origin = (0.0, 0.0)
        xy = np.array([[0.5 - dx * h, 0.5 - dy * h]])  # cell (0,0) centre at (0.5, 0.5)
        out.append(oracle.kde_grid(xy, None, origin, 1.0, 1, 1, h, oracle.RADIAL + kid)[0, 0])
    return np.array(out)


@pytest.mark.parametrize("kid", COMPACT, ids=[oracle.KERNEL_NAMES[k] for k in COMPACT])
def test_radial_symmetry_and_disk_support(kid):
    r = 0.6
    angles = np.linspace(0.0, 2 * math.pi, 7, endpoint=False)
    F = _single_point_density(kid, [(r * math.cos(a), r * math.sin(a)) for a in angles])
    assert F[0] > 0
    np.testing.assert_allclose(F, F[0], rtol=1e-12)
    # corner of the square support: inside for the product kernel, outside the disk
    out = _single_point_density(kid, [(0.8, 0.8)])[0]
    assert out == 0.0
    product = oracle.kde_grid(np.array([[0.5 - 0.8, 0.5 - 0.8]]), None, (0.0, 0.0), 1.0, 1, 1,
                              1.0, kid)[0, 0]
    assert product > 0.0


def test_radial_gaussian_is_the_product_gaussian():
    rng = np.random.default_rng(5)
    xy = rng.uniform(0, 100, (50, 2))
    w = rng.uniform(0.5, 2.0, 50)
    a = oracle.kde_grid(xy, w, (0.0, 0.0), 5.0, 20, 20, 12.0, oracle.GAUSSIAN)
    b = oracle.kde_grid(xy, w, (0.0, 0.0), 5.0, 20, 20, 12.0, oracle.RADIAL + oracle.GAUSSIAN)
    np.testing.assert_allclose(b, a, rtol=1e-13, atol=0)


def test_radial_density_mass_on_a_fine_grid():
    """Midpoint rule over the grid: cell^2 sum F -> sum w / N as cell/h -> 0
    (the density is normalised over the plane, support inside the grid)."""
    for kid in (oracle.EPANECHNIKOV, oracle.TRIWEIGHT, oracle.COSINE):
        xy = np.array([[50.3, 49.8], [47.0, 52.5]])
        F = oracle.kde_grid(xy, np.array([1.0, 3.0]), (0.0, 0.0), 0.25, 400, 400, 20.0,
                            oracle.RADIAL + kid)
        assert abs(0.25 ** 2 * F.sum() - 2.0) < 2e-4
