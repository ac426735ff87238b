"""The synthetic inputs have the structure their recipe states (CPU only):
vessels at 5-20 kn with a fix every 10 s, the jitter asked for, the lane /
port / background mix of the 20M-point workload, the batched instances'
parameter ranges, and seeded determinism.  Reduced trajectory counts keep it
fast; the generators are the ones the full sizes use."""
import math

import numpy as np
import pytest

import workloads as W

KN = 1852.0 / 3600.0


def _steps(local, fixes):
    t = local.reshape(-1, fixes, 2)
    return np.hypot(*np.diff(t, axis=1).transpose(2, 0, 1))


def test_lane_speeds_and_fix_interval():
    """Without jitter a step between fixes is a chord of speed x 10 s of arc:
    never longer than 20 kn x 10 s, and typically between 5 and 20 kn."""
    rng = np.random.default_rng(11)
    local = W.lane_traffic(rng, 60, 200, 50_000.0, 4, jitter=0.0)
    st = _steps(local, 200)
    assert st.max() <= 20 * KN * 10 + 1e-6
    med = np.median(st, axis=1)
    assert med.min() >= 0.95 * 5 * KN * 10 and med.max() <= 20 * KN * 10 + 1e-6
    # speeds spread over the range, not one value
    assert med.max() - med.min() > 0.5 * 15 * KN * 10


def test_lane_jitter_is_the_requested_sigma():
    a = W.lane_traffic(np.random.default_rng(12), 40, 300, 50_000.0, 4, jitter=0.0)
    b = W.lane_traffic(np.random.default_rng(12), 40, 300, 50_000.0, 4, jitter=20.0)
    d = b - a
    assert abs(d.mean()) < 0.5
    assert d.std() == pytest.approx(20.0, rel=0.03)


def test_mixture_workload_structure():
    """The 20M-point recipe at 200 trajectories: 70% lane, 20% port, 10%
    uniform trajectories of 500 fixes, in that order."""
    wl = W.config3(n_traj=200, grid=1024)
    assert wl.n == 200 * 500 and wl.nx == wl.ny == 1024
    assert wl.cell == pytest.approx(100_000.0 / 1024) and wl.h == 100.0
    assert np.array_equal(wl.offsets, np.arange(201) * 500)
    t = wl.local.reshape(200, 500, 2)
    lane, port, uni = t[:140], t[140:180], t[180:]
    # lanes: steps of a 5-20 kn vessel plus 20 m jitter on each end
    med = np.median(np.hypot(*np.diff(lane, axis=1).transpose(2, 0, 1)), axis=1)
    assert med.min() > 20.0 and med.max() < 20 * KN * 10 + 60.0
    # ports: each trajectory is one port's cluster of sigma 500 m
    sd = port.std(axis=1)
    assert np.all((sd > 400.0) & (sd < 600.0))
    # background: uniform over the box
    u = uni.reshape(-1, 2)
    assert u.min() >= 0.0 and u.max() <= 100_000.0
    assert u.mean(0) == pytest.approx([50_000.0, 50_000.0], rel=0.03)
    assert u.std(0) == pytest.approx([100_000.0 / math.sqrt(12)] * 2, rel=0.03)


def test_lane_workload_stays_in_its_box():
    wl = W.config2(n_traj=200)
    assert wl.n == 100_000 and wl.box == 50_000.0 and wl.h == 150.0
    inside = np.all((wl.local >= 0) & (wl.local <= wl.box), axis=1)
    assert inside.mean() > 0.99


def test_batched_instances_parameter_ranges():
    inst = W.config4_instances(count=256, n_range=(1000, 3000))
    assert len(inst) == 256
    sides = {x.nx for x in inst}
    assert sides <= {128, 256, 512, 1024, 2048} and len(sides) == 5
    assert all(x.nx == x.ny and x.cell == pytest.approx(x.box / x.nx) for x in inst)
    assert all(50.0 <= x.h <= 800.0 and 10_000.0 <= x.box <= 100_000.0 for x in inst)
    assert all(1000 <= x.n <= 3000 and x.local.shape == (x.n, 2) for x in inst)
    gauss = sum(x.kernel == W.GAUSSIAN for x in inst)
    assert {x.kernel for x in inst} == {W.GAUSSIAN, W.EPANECHNIKOV}
    assert 0.4 < gauss / 256 < 0.6


def test_small_lane_case_geometry():
    wl = W.config1()
    assert wl.n == 2000 and wl.nx * wl.cell == wl.box == 20_000.0
    assert np.array_equal(wl.offsets, np.arange(21) * 100)
    assert np.all(wl.w == 1.0)


def test_lonlat_box_is_centred_on_the_reference_point():
    wl = W.config1()
    _, corner, lat_c = wl.lonlat()
    centre = W.Workload("c", np.array([[wl.box / 2, wl.box / 2]]), np.ones(1, np.float32),
                        wl.box, wl.cell, 1, 1, wl.h, wl.kernel, np.array([0, 1]), 0)
    c_ll, _, _ = centre.lonlat()
    assert c_ll[0] == pytest.approx([W.REF_LON, W.REF_LAT], abs=1e-12)
    assert corner[0] < W.REF_LON and corner[1] < W.REF_LAT and lat_c == W.REF_LAT
    # absolute metres are the local ones shifted by the false origin (to the
    # rounding of a 1.4e7 m sum, 2^-29 m)
    assert np.allclose(wl.xy - np.asarray(W.FALSE_ORIGIN), wl.local, rtol=0, atol=4e-9)


def test_seeded_and_repeatable():
    a, b = W.config2(n_traj=50), W.config2(n_traj=50)
    assert np.array_equal(a.local, b.local)
    c = W.config2(seed=7, n_traj=50)
    assert not np.array_equal(a.local, c.local)
