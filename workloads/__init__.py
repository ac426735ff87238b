"""Seeded synthetic AIS-like inputs shared by the tests, the bench and smoke().

This module holds none of the method's arithmetic (no kernel, no projection,
no density): it only draws positions.  The paper's three AIS datasets
(Sec. V, Table 3) are not available, so these stand in for them, with the
shapes and structure of its workloads: vessels following shipping lanes at
5-20 kn with AIS fixes every 10 s, clusters around ports, and a uniform
background, in boxes of 20-100 km.

Positions are drawn in local metres inside the box and returned two ways:
  * ``xy``: absolute metres = local metres + a large false origin (so that the
    library's FP64 centring step is exercised), with ``origin`` = the grid's
    lower-left corner in the same frame;
  * ``lonlat``: degrees around the centre of the paper's Yangtze South Channel
    box, converted with a plain equirectangular scale (mean Earth radius); the
    library and the oracle each apply the paper's Mercator projection to these.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# centre of the Yangtze South Channel box of Table 3 (degrees)
REF_LON = 0.5 * (121.3795 + 121.9842)
REF_LAT = 0.5 * (31.5746 + 31.1166)
MEAN_EARTH_RADIUS = 6371008.8
KNOT = 1852.0 / 3600.0
# false origin of the absolute-metre frame (magnitude of projected coordinates)
FALSE_ORIGIN = (13_545_000.0, 3_652_000.0)

GAUSSIAN, EPANECHNIKOV = 6, 2


@dataclasses.dataclass
class Workload:
    name: str
    local: np.ndarray            # [n,2] float64 metres inside the box
    w: np.ndarray                # [n] float32 weights
    box: float                   # side of the square box, metres
    cell: float                  # grid cell side, metres
    nx: int
    ny: int
    h: float                     # bandwidth, metres
    kernel: int                  # Table 1 kernel id
    offsets: np.ndarray          # [ntraj+1] trajectory boundaries
    seed: int

    @property
    def n(self) -> int:
        return int(self.local.shape[0])

    @property
    def origin(self):
        return FALSE_ORIGIN

    @property
    def xy(self) -> np.ndarray:
        """Absolute metres, interleaved [n,2] float64."""
        out = self.local.copy()
        out[:, 0] += FALSE_ORIGIN[0]
        out[:, 1] += FALSE_ORIGIN[1]
        return out

    def lonlat(self) -> tuple[np.ndarray, tuple[float, float], float]:
        """(lon,lat) degrees [n,2], the box's lower-left corner, and the
        standard latitude (box centre) for the projection."""
        lat_c = REF_LAT
        k_lat = 180.0 / (math.pi * MEAN_EARTH_RADIUS)
        k_lon = k_lat / math.cos(math.radians(lat_c))
        lon0 = REF_LON - 0.5 * self.box * k_lon
        lat0 = lat_c - 0.5 * self.box * k_lat
        ll = np.empty_like(self.local)
        ll[:, 0] = lon0 + self.local[:, 0] * k_lon
        ll[:, 1] = lat0 + self.local[:, 1] * k_lat
        return ll, (lon0, lat0), lat_c


# ---------------------------------------------------------------- primitives

def _polyline_positions(way: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Points at arc lengths s (clipped by reflection) along a polyline."""
    seg = np.diff(way, axis=0)
    seglen = np.hypot(seg[:, 0], seg[:, 1])
    cum = np.concatenate([[0.0], np.cumsum(seglen)])
    total = cum[-1]
    # reflect arc lengths into [0, total] (a vessel turning back at the end)
    period = 2.0 * total
    s = np.mod(s, period)
    s = np.where(s > total, period - s, s)
    x = np.interp(s, cum, way[:, 0])
    y = np.interp(s, cum, way[:, 1])
    return np.stack([x, y], axis=-1)


def _waypoint_graph(rng: np.random.Generator, box: float, k: int) -> np.ndarray:
    """A lane: k waypoints crossing the box, chained in order of progress."""
    a = rng.uniform(0.0, 2.0 * math.pi)
    d = np.array([math.cos(a), math.sin(a)])
    c = np.array([0.5 * box, 0.5 * box]) + rng.uniform(-0.2, 0.2, 2) * box
    t = np.linspace(-0.55, 0.55, k) * box
    pts = c[None, :] + t[:, None] * d[None, :]
    perp = np.array([-d[1], d[0]])
    pts += perp[None, :] * rng.normal(0.0, 0.08 * box, (k, 1))
    return np.clip(pts, 0.02 * box, 0.98 * box)


def lane_traffic(rng, n_traj: int, fixes: int, box: float, n_graphs: int,
                 jitter: float, dt: float = 10.0, kn=(5.0, 20.0),
                 lane_sigma: float = 60.0):
    """Vessels on lanes: speed U(kn) knots, one fix every dt seconds."""
    graphs = [_waypoint_graph(rng, box, 6) for _ in range(n_graphs)]
    gid = rng.integers(0, n_graphs, n_traj)
    speed = rng.uniform(kn[0], kn[1], n_traj) * KNOT
    direction = rng.choice([-1.0, 1.0], n_traj)
    start = rng.uniform(0.0, 2.0 * box, n_traj)
    lateral = rng.normal(0.0, lane_sigma, n_traj)
    k = np.arange(fixes, dtype=np.float64)
    out = np.empty((n_traj, fixes, 2))
    for g, way in enumerate(graphs):
        sel = np.nonzero(gid == g)[0]
        if sel.size == 0:
            continue
        s = start[sel, None] + direction[sel, None] * speed[sel, None] * dt * k[None, :]
        pos = _polyline_positions(way, s.ravel()).reshape(sel.size, fixes, 2)
        seg = way[-1] - way[0]
        nrm = np.array([-seg[1], seg[0]]) / max(np.hypot(seg[0], seg[1]), 1e-9)
        pos += lateral[sel, None, None] * nrm[None, None, :]
        out[sel] = pos
    out += rng.normal(0.0, jitter, out.shape)
    return out.reshape(-1, 2)


def port_clusters(rng, n_traj: int, fixes: int, box: float, n_ports: int, sigma: float):
    ports = rng.uniform(0.1 * box, 0.9 * box, (n_ports, 2))
    pid = rng.integers(0, n_ports, n_traj)
    pts = ports[pid][:, None, :] + rng.normal(0.0, sigma, (n_traj, fixes, 2))
    return pts.reshape(-1, 2)


def uniform_background(rng, n_traj: int, fixes: int, box: float):
    return rng.uniform(0.0, box, (n_traj * fixes, 2))


def _offsets(n_traj: int, fixes: int) -> np.ndarray:
    return np.arange(n_traj + 1, dtype=np.int64) * fixes


# -------------------------------------------------------------- the configs

def config1(seed: int = 1001) -> Workload:
    """20 vessels x 100 fixes on seeded piecewise-linear lanes, 20 km box,
    30 m jitter, unit weights; 64x64 grid of 312.5 m cells, h = 200 m."""
    rng = np.random.default_rng(seed)
    box = 20_000.0
    tracks = []
    for _ in range(20):
        way = rng.uniform(0.05 * box, 0.95 * box, (rng.integers(2, 5), 2))
        seg = np.hypot(*np.diff(way, axis=0).T).sum()
        s = np.linspace(0.0, seg, 100)
        tracks.append(_polyline_positions(way, s))
    local = np.concatenate(tracks) + rng.normal(0.0, 30.0, (2000, 2))
    return Workload("gaussian 2k pts, 64x64 grid, h=200 m", local,
                    np.ones(2000, np.float32), box, 312.5, 64, 64, 200.0,
                    GAUSSIAN, _offsets(20, 100), seed)


def config2(seed: int = 1002, n_traj: int = 2000, fixes: int = 500,
            kernel: int = GAUSSIAN) -> Workload:
    """2000 trajectories x 500 fixes (1M points) on lanes of 8 waypoint graphs,
    5-20 kn, 10 s fixes, 20 m jitter, 50 km box; 1024^2 grid, h = 150 m."""
    rng = np.random.default_rng(seed)
    box = 50_000.0
    local = lane_traffic(rng, n_traj, fixes, box, 8, 20.0)
    n = local.shape[0]
    return Workload(f"{n} pts lanes, 1024^2 grid, h=150 m", local,
                    np.ones(n, np.float32), box, box / 1024, 1024, 1024, 150.0,
                    kernel, _offsets(n_traj, fixes), seed)


def config3(seed: int = 1003, n_traj: int = 40_000, fixes: int = 500,
            grid: int = 4096) -> Workload:
    """40,000 trajectories x 500 fixes (20M points): 70% lane traffic, 20% port
    clusters (sigma 500 m around 20 ports), 10% uniform; 100 km box;
    4096^2 grid (24.4140625 m cells), h = 100 m, Gaussian."""
    rng = np.random.default_rng(seed)
    box = 100_000.0
    n_lane = int(round(0.7 * n_traj))
    n_port = int(round(0.2 * n_traj))
    n_uni = n_traj - n_lane - n_port
    parts = [lane_traffic(rng, n_lane, fixes, box, 12, 20.0),
             port_clusters(rng, n_port, fixes, box, 20, 500.0),
             uniform_background(rng, n_uni, fixes, box)]
    local = np.concatenate(parts)
    n = local.shape[0]
    return Workload(f"{n} pts mixture, {grid}^2 grid, h=100 m", local,
                    np.ones(n, np.float32), box, box / grid, grid, grid, 100.0,
                    GAUSSIAN, _offsets(n_traj, fixes), seed)


def config4_instances(seed: int = 1004, count: int = 256, n_range=(1e4, 2e6),
                      side_pow=(7, 11)):
    """Batched: point counts log-uniform in n_range, grid side 2^U{side_pow},
    h ~ U(50, 800) m, Gaussian/Epanechnikov 50/50, box side U(10, 100) km."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1]))))
        side = 2 ** int(rng.integers(side_pow[0], side_pow[1] + 1))
        h = float(rng.uniform(50.0, 800.0))
        kern = GAUSSIAN if rng.random() < 0.5 else EPANECHNIKOV
        box = float(rng.uniform(10_000.0, 100_000.0))
        fixes = 500
        n_traj = max(1, n // fixes)
        n_lane = max(1, int(0.7 * n_traj))
        pts = [lane_traffic(rng, n_lane, fixes, box, 4, 20.0)]
        rest = n - n_lane * fixes
        if rest > 0:
            pts.append(port_clusters(rng, 1, rest, box, 3, 0.01 * box))
        local = np.concatenate(pts)[:n]
        out.append(Workload(f"instance {k}", local, np.ones(n, np.float32), box,
                            box / side, side, side, h, kern,
                            np.array([0, n], dtype=np.int64), seed * 1000 + k))
    return out


def config5_raw(seed: int = 1005, n_traj: int = 4000, fixes: int = 500) -> Workload:
    """2M points from the lane generator (to be thinned by Douglas-Peucker at
    eps = 10 m); 1024^2 grid over a 50 km box, initial h = 150 m."""
    return config2(seed=seed, n_traj=n_traj, fixes=fixes)


def random_points(seed: int, n: int, box: float, cell: float, nx: int, ny: int, h: float,
                  kernel: int, weighted: bool = True) -> Workload:
    """Small uniform cases for parity tests (weights U(0.5, 2) when weighted)."""
    rng = np.random.default_rng(seed)
    local = rng.uniform(-0.1 * box, 1.1 * box, (n, 2))
    w = (rng.uniform(0.5, 2.0, n) if weighted else np.ones(n)).astype(np.float32)
    return Workload(f"uniform {n} pts", local, w, box, cell, nx, ny, h, kernel,
                    np.array([0, n], dtype=np.int64), seed)
