"""The work counts bench.py divides by time (CPU only): the evaluated pairs of
the cutoff path and the point-tile products of the block-sparse contraction.
Each is bracketed by brute-force counts over every output block or tile:
from below by the points within the exact reach of the block's cell centres
(every pair the method needs), from above by the same count with the reach
widened by one sort bin and one more reach (the bin granularity and the
clipping of outside points into the edge bins); and the prefix sums over the
bin histograms equal a brute-force loop over blocks and points.  A dropped
block, a wrong reach or scale, a transposed axis or a count of all points
fails one of them."""
import math

import numpy as np
import pytest

import bench


def _points(seed, n, nx, ny, cell, out=0.2):
    """Uniform points over the grid and a margin of `out` of its size around it."""
    rng = np.random.default_rng(seed)
    W, H = nx * cell, ny * cell
    x = rng.uniform(-out * W, (1 + out) * W, n)
    y = rng.uniform(-out * H, (1 + out) * H, n)
    return np.stack([x, y], 1)


def _per_block(X, Y, nx, ny, B, cs, reach):
    """Sum over B x B-cell blocks of the points within `reach` (per axis) of
    the block's span of cell centres, all in the units X, Y are in."""
    total = 0
    for j0 in range(0, ny, B):
        ylo, yhi = (j0 + 0.5) * cs - reach, (min(j0 + B, ny) - 0.5) * cs + reach
        iny = (Y >= ylo) & (Y <= yhi)
        for i0 in range(0, nx, B):
            xlo, xhi = (i0 + 0.5) * cs - reach, (min(i0 + B, nx) - 0.5) * cs + reach
            total += int(np.count_nonzero(iny & (X >= xlo) & (X <= xhi)))
    return total


def _support_pairs(X, Y, nx, ny, cs):
    """Point-cell pairs with |s| <= 1 and |t| <= 1 (units of h)."""
    gx = (np.arange(nx) + 0.5) * cs
    gy = (np.arange(ny) + 0.5) * cs
    sx = (np.abs(gx[None, :] - X[:, None]) <= 1).sum(1)
    sy = (np.abs(gy[None, :] - Y[:, None]) <= 1).sum(1)
    return int((sx * sy).sum())


@pytest.mark.parametrize("nx,ny,h_cells,n", [(40, 40, 2.0, 300), (53, 37, 0.7, 500),
                                              (96, 64, 9.0, 200), (70, 90, 20.0, 150)])
def test_cutoff_pairs_bracketed(nx, ny, h_cells, n):
    cell = 10.0
    h = h_cells * cell
    xy = _points(nx + ny, n, nx, ny, cell)
    got = bench.cutoff_pairs(xy, (0.0, 0.0), cell, nx, ny, h)
    cs = cell / h
    X, Y = xy[:, 0] / h, xy[:, 1] / h
    S = 4 if h_cells <= 6 else 8 if h_cells <= 16 else 16
    lower = 256 * _per_block(X, Y, nx, ny, 16, cs, 1.0)
    upper = 256 * _per_block(X, Y, nx, ny, 16, cs, 2.0 + S * cs)
    assert lower <= got <= upper
    # every support pair is among the evaluated ones, and no block reads more
    # than all the points
    assert got >= _support_pairs(X, Y, nx, ny, cs)
    assert got <= 256 * n * math.ceil(nx / 16) * math.ceil(ny / 16)


@pytest.mark.parametrize("nx,ny,h_cells,n", [(512, 512, 1.5, 400), (300, 700, 4.0, 300),
                                              (1024, 256, 0.8, 500)])
def test_sparse_products_bracketed(nx, ny, h_cells, n):
    cell = 10.0
    h = h_cells * cell
    xy = _points(nx * 3 + ny, n, nx, ny, cell)
    got = bench.sparse_products(xy, (0.0, 0.0), cell, nx, ny, h)
    sigma = 1.0 / (h * math.sqrt(2.0 * math.log(2.0)))
    cs = cell * sigma
    X, Y = xy[:, 0] * sigma, xy[:, 1] * sigma
    reach = 6.45
    lower = _per_block(X, Y, nx, ny, 256, cs, reach)
    upper = _per_block(X, Y, nx, ny, 256, cs, 2 * reach + 32 * cs)
    assert lower <= got <= upper
    assert got <= n * math.ceil(nx / 256) * math.ceil(ny / 256)


def _bin_reads(X, Y, nx, ny, B, cs, S, reach, keep_reach):
    """Brute force over blocks and points: the points whose sort bin (S cells,
    edge bins taking the points outside the grid but within `keep_reach` of
    it) lies in the bins a B x B-cell block's cell centres reach."""
    inv_binw = 1.0 / (S * cs)
    nbx, nby = -(-nx // S), -(-ny // S)
    keep = ((X >= -keep_reach) & (Y >= -keep_reach) & (X <= nx * cs + keep_reach)
            & (Y <= ny * cs + keep_reach))
    bx = [min(max(math.floor(x * inv_binw), 0), nbx - 1) for x in X[keep]]
    by = [min(max(math.floor(y * inv_binw), 0), nby - 1) for y in Y[keep]]
    total = 0
    for j0 in range(0, ny, B):
        ly = max(0, math.floor(((j0 + 0.5) * cs - reach) * inv_binw))
        hy = min(nby - 1, math.floor(((j0 + B - 0.5) * cs + reach) * inv_binw))
        for i0 in range(0, nx, B):
            lx = max(0, math.floor(((i0 + 0.5) * cs - reach) * inv_binw))
            hx = min(nbx - 1, math.floor(((i0 + B - 0.5) * cs + reach) * inv_binw))
            total += sum(1 for a, b in zip(bx, by) if lx <= a <= hx and ly <= b <= hy)
    return total


@pytest.mark.parametrize("nx,ny,h_cells,n", [(40, 40, 2.0, 300), (53, 37, 0.7, 500),
                                              (96, 64, 9.0, 200), (70, 90, 20.0, 150)])
def test_cutoff_pairs_equal_brute_force(nx, ny, h_cells, n):
    """The prefix sums over the bin histogram equal a per-block loop over the
    points' bins (16 x 16-cell blocks, 256 cells each)."""
    cell = 10.0
    h = h_cells * cell
    xy = _points(nx + ny, n, nx, ny, cell)
    cs = cell / h
    S = 4 if h_cells <= 6 else 8 if h_cells <= 16 else 16
    reach = 1.0 + 1e-6 + 8.0 * 2.0 ** -24 * (max(nx, ny) * cs + 1.0)
    want = 256 * _bin_reads(xy[:, 0] / h, xy[:, 1] / h, nx, ny, 16, cs, S, reach, 1.0)
    assert bench.cutoff_pairs(xy, (0.0, 0.0), cell, nx, ny, h) == want


@pytest.mark.parametrize("nx,ny,h_cells,n", [(512, 512, 1.5, 400), (300, 700, 4.0, 300),
                                              (1024, 256, 0.8, 500)])
def test_sparse_products_equal_brute_force(nx, ny, h_cells, n):
    """Likewise for the 256 x 256 tiles over 32 x 32-cell bins, in units of
    h sqrt(2 ln 2)."""
    cell = 10.0
    h = h_cells * cell
    xy = _points(nx * 3 + ny, n, nx, ny, cell)
    sigma = 1.0 / (h * math.sqrt(2.0 * math.log(2.0)))
    cs = cell * sigma
    reach = 6.45 + 1e-6 + 8.0 * 2.0 ** -24 * (max(nx, ny) * cs + 6.45)
    want = _bin_reads(xy[:, 0] * sigma, xy[:, 1] * sigma, nx, ny, 256, cs, 32, reach, reach)
    assert bench.sparse_products(xy, (0.0, 0.0), cell, nx, ny, h) == want


def test_sparse_reach_drops_only_negligible_terms():
    """The reach in units of h sqrt(2 ln 2): a factor past it is 2^-(6.45^2),
    below 2^-41, far under FP16's smallest subnormal relative to a peak of 1."""
    assert 2.0 ** -(6.45 ** 2) < 2.0 ** -41
    assert math.exp(-0.5 * (6.45 * math.sqrt(2 * math.log(2))) ** 2) == pytest.approx(
        2.0 ** -(6.45 ** 2), rel=1e-12)


def test_measured_traffic_follows_the_source_hash(monkeypatch):
    key = ("tc_split16", 4096, 40_000)
    entry = dict(bench.TRAFFIC[key])
    monkeypatch.setitem(bench.TRAFFIC, key, dict(entry, sha256="0" * 64))
    assert bench.measured_traffic(*key) is None
    import hashlib
    hsh = hashlib.sha256()
    for f in entry["sources"]:
        with open(f"{bench.ROOT}/{f}", "rb") as fh:
            hsh.update(fh.read())
    monkeypatch.setitem(bench.TRAFFIC, key, dict(entry, sha256=hsh.hexdigest()))
    assert bench.measured_traffic(*key) == entry["bytes"]
    assert bench.measured_traffic("tc_split16", 2048, 40_000) is None


@pytest.mark.parametrize("nx,ny,h_cells,n", [(40, 40, 2.0, 300), (53, 37, 0.7, 500),
                                              (96, 64, 9.0, 200), (70, 90, 20.0, 150)])
def test_support_pairs_equal_brute_force(nx, ny, h_cells, n):
    """The cutoff path's algorithmic work: every point against every cell,
    counting the pairs with both offsets within a bandwidth."""
    cell = 10.0
    h = h_cells * cell
    xy = _points(nx + ny + 7, n, nx, ny, cell)
    cs = cell / h
    want = _support_pairs(xy[:, 0] / h, xy[:, 1] / h, nx, ny, cs)
    assert bench.support_pairs(xy, (0.0, 0.0), cell, nx, ny, h) == want
