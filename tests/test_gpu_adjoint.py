"""Adjoint of the Gaussian density, the grid LSCV loss and the bandwidth fit,
through the C ABI, against the FP64 oracle's analytic gradients (relative
L-inf within 1e-4, normalised by the largest oracle component)."""
import math

import numpy as np
import pytest

import oracle
import workloads
from kde_testutil import TOL_GRAD, rel_linf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2004_13653_gb300 as kde  # noqa: E402
from paper_2004_13653_gb300 import autograd as kag  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kde.load(build_if_stale=True)


def _dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _case(seed=900, n=300, nx=60, ny=50):
    wl = workloads.random_points(seed, n, 600.0, 10.0, nx, ny, 25.0, oracle.GAUSSIAN)
    G = np.random.default_rng(seed).normal(0, 1, (ny, nx))
    return wl, G


def test_adjoint_matches_oracle_vjp():
    wl, G = _case()
    gxy, gw, gh = kde.grid_backward(_dev(wl.xy, torch.float64), _dev(wl.w, torch.float32),
                                    wl.origin, wl.cell, wl.nx, wl.ny, wl.h,
                                    _dev(G, torch.float32))
    rw, rxy, rh = oracle.kde_vjp_gauss(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, G)
    assert rel_linf(gw.cpu().numpy(), rw) <= TOL_GRAD
    assert rel_linf(gxy.cpu().numpy(), rxy) <= TOL_GRAD
    # each component of at least a tenth of the largest, against itself
    assert _rel_per_point(gw.cpu().numpy(), rw) <= 10 * TOL_GRAD
    assert _rel_per_point(gxy.cpu().numpy(), rxy) <= 10 * TOL_GRAD
    assert gh == pytest.approx(rh, rel=TOL_GRAD)


def test_adjoint_wide_bandwidth_whole_grid_window():
    """h = 40 cells: the +-8h window covers the whole grid."""
    wl = workloads.random_points(901, 200, 300.0, 5.0, 60, 60, 200.0, oracle.GAUSSIAN)
    G = np.random.default_rng(901).normal(0, 1, (60, 60))
    gxy, gw, gh = kde.grid_backward(_dev(wl.xy, torch.float64), _dev(wl.w, torch.float32),
                                    wl.origin, wl.cell, 60, 60, wl.h, _dev(G, torch.float32))
    rw, rxy, rh = oracle.kde_vjp_gauss(wl.xy, wl.w, wl.origin, wl.cell, 60, 60, wl.h, G)
    assert rel_linf(gw.cpu().numpy(), rw) <= TOL_GRAD
    assert rel_linf(gxy.cpu().numpy(), rxy) <= TOL_GRAD
    assert gh == pytest.approx(rh, rel=TOL_GRAD)


@pytest.mark.parametrize("h_cells,n", [(0.1, 7), (0.3, 300), (0.7, 333), (1.2, 65), (1.7, 301)])
def test_adjoint_narrow_windows(h_cells, n):
    """Windows of 5, 9, 15, 23 and 31 columns: at most 16 columns take 32 / 2^k
    rows at a time (2^k >= width lanes per row); batches of 32 points per warp
    end ragged (7, 333, 65 and 301 points; the seeds keep the h-term's
    cancellation below 100x)."""
    wl = workloads.random_points(902 + n, n, 600.0, 10.0, 60, 50, 10.0 * h_cells,
                                 oracle.GAUSSIAN)
    G = np.random.default_rng(902).normal(0, 1, (50, 60))
    gxy, gw, gh = kde.grid_backward(_dev(wl.xy, torch.float64), _dev(wl.w, torch.float32),
                                    wl.origin, wl.cell, 60, 50, wl.h, _dev(G, torch.float32))
    rw, rxy, rh = oracle.kde_vjp_gauss(wl.xy, wl.w, wl.origin, wl.cell, 60, 50, wl.h, G)
    assert rel_linf(gw.cpu().numpy(), rw) <= TOL_GRAD
    assert rel_linf(gxy.cpu().numpy(), rxy) <= TOL_GRAD
    assert _rel_per_point(gw.cpu().numpy(), rw) <= 10 * TOL_GRAD
    assert _rel_per_point(gxy.cpu().numpy(), rxy) <= 10 * TOL_GRAD
    assert gh == pytest.approx(rh, rel=TOL_GRAD)


def test_lscv_loss_cotangent_and_direct_terms_match_oracle():
    wl, _ = _case(902, 400)
    F = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, oracle.GAUSSIAN)
    loss, G, gw, gxy, gh = kde.lscv_grid(_dev(F, torch.float32), _dev(wl.xy, torch.float64),
                                         _dev(wl.w, torch.float32), wl.origin, wl.cell, wl.nx,
                                         wl.ny, wl.h)
    ref_loss = oracle.lscv_loss(F, wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h)
    ref_G = oracle.lscv_cotangent(F, wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny)
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    assert rel_linf(G.cpu().numpy(), ref_G) <= 1e-5


def test_lscv_gradient_through_autograd_matches_oracle():
    """dL/d(log h) and dL/domega (w = N softmax(omega)) from the GPU chain
    (split-FP16 forward, adjoint, LSCV) against the oracle's FP64 analytic
    gradient, itself pinned to central differences."""
    wl, _ = _case(903, 500, 64, 64)
    n = wl.n
    omega0 = np.log(wl.w.astype(np.float64) / wl.w.sum())
    log_h = torch.tensor(math.log(wl.h), dtype=torch.float64, device="cuda", requires_grad=True)
    omega = torch.tensor(omega0, dtype=torch.float64, device="cuda", requires_grad=True)
    pts = _dev(wl.xy, torch.float64)
    w = (n * torch.softmax(omega, 0)).to(torch.float32)
    L = kag.lscv_loss(pts, w, torch.exp(log_h), wl.origin, wl.cell, wl.nx, wl.ny)
    L.backward()
    wv = n * np.exp(omega0) / np.exp(omega0).sum()
    rL, rgw, rgxy, rgh = oracle.lscv_value_and_grad(wl.xy, wv, wl.origin, wl.cell, wl.nx, wl.ny,
                                                    wl.h)
    assert float(L) == pytest.approx(rL, rel=1e-4)
    assert float(log_h.grad) == pytest.approx(wl.h * rgh, rel=TOL_GRAD, abs=1e-4 * abs(wl.h * rgh))
    ref_om = wv * (rgw - np.sum(wv * rgw) / n)
    assert rel_linf(omega.grad.cpu().numpy(), ref_om) <= TOL_GRAD


def test_config5_adjoint_sampled_points():
    """2M lane fixes thinned by the oracle's Douglas-Peucker at 10 m, 1024^2
    grid, h = 150 m, cotangent = the LSCV cotangent: the adjoint on sampled
    points against the oracle."""
    raw = workloads.config5_raw()
    keep = oracle.douglas_peucker(raw.local, raw.offsets, 10.0)
    xy = raw.xy[keep]
    w = np.ones(xy.shape[0], np.float32)
    F = kde.grid(_dev(xy, torch.float64), _dev(w, torch.float32), raw.origin, raw.cell, raw.nx,
                 raw.ny, raw.h, "gaussian", flags=kde.FLAG_SYNC)
    loss, G, _, _, _ = kde.lscv_grid(F, _dev(xy, torch.float64), _dev(w, torch.float32),
                                     raw.origin, raw.cell, raw.nx, raw.ny, raw.h)
    gxy, gw, _ = kde.grid_backward(_dev(xy, torch.float64), _dev(w, torch.float32), raw.origin,
                                   raw.cell, raw.nx, raw.ny, raw.h, G, want_h=False)
    sel = np.random.default_rng(5).choice(xy.shape[0], 48, replace=False)
    rw, rxy, _ = oracle.kde_vjp_gauss(xy, w, raw.origin, raw.cell, raw.nx, raw.ny, raw.h,
                                      G.cpu().numpy().astype(np.float64), pts=sel)
    assert rel_linf(gw.cpu().numpy()[sel], rw) <= TOL_GRAD
    assert rel_linf(gxy.cpu().numpy()[sel], rxy) <= TOL_GRAD


def test_fit_bandwidth_decreases_loss_and_resumes(tmp_path):
    wl = workloads.config2(seed=904, n_traj=20, fixes=500)
    wl.nx = wl.ny = 256
    wl.cell = wl.box / 256
    pts = _dev(wl.xy, torch.float64)
    w0 = torch.ones(wl.n, dtype=torch.float32, device="cuda")
    h_full, w_full, losses = kag.fit_bandwidth(pts, w0, wl.origin, wl.cell, 256, 256, 150.0,
                                               steps=40, lr=0.05)
    assert losses[-1] < losses[0]
    ck = str(tmp_path / "lscv.pt")
    kag.fit_bandwidth(pts, w0, wl.origin, wl.cell, 256, 256, 150.0, steps=20, lr=0.05,
                      checkpoint=ck, every=10)
    h_res, w_res, losses_res = kag.fit_bandwidth(pts, w0, wl.origin, wl.cell, 256, 256, 150.0,
                                                 steps=40, lr=0.05, checkpoint=ck, every=10)
    assert len(losses_res) == 40
    assert h_res == pytest.approx(h_full, rel=1e-6)
    assert losses_res[-1] == pytest.approx(losses[-1], rel=1e-6)


def _rel_per_point(got, ref, floor=0.1):
    """Largest error relative to each component itself, over the components
    whose size is at least `floor` of the largest (small-gradient points are
    checked by the L-inf test, where the largest component normalises)."""
    got = np.asarray(got, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    big = np.abs(ref) >= floor * np.max(np.abs(ref))
    return float(np.max(np.abs(got[big] - ref[big]) / np.abs(ref[big])))


@pytest.mark.parametrize("path", ["simt", "tc_split16"])
def test_both_adjoint_forms_match_oracle(path):
    """The window kernel and the two tensor-core contractions, forced, on the
    same case: dL/dw, dL/dpoints and dL/dh against the oracle's VJP."""
    wl, G = _case(seed=905, n=777, nx=300, ny=130)
    gxy, gw, gh = kde.grid_backward(_dev(wl.xy, torch.float64), _dev(wl.w, torch.float32),
                                    wl.origin, wl.cell, wl.nx, wl.ny, wl.h,
                                    _dev(G, torch.float32), path=path)
    rw, rxy, rh = oracle.kde_vjp_gauss(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, G)
    assert rel_linf(gw.cpu().numpy(), rw) <= TOL_GRAD
    assert rel_linf(gxy.cpu().numpy(), rxy) <= TOL_GRAD
    assert _rel_per_point(gxy.cpu().numpy(), rxy) <= 10 * TOL_GRAD
    assert gh == pytest.approx(rh, rel=TOL_GRAD)


def test_contraction_adjoint_wide_bandwidth_large_grid():
    """h = 16 cells on a 520 x 540 grid (ragged 256-cell tiles and 64-cell
    stages), 2001 points partly outside the grid: the contractions (AUTO picks
    them here) against the oracle's VJP on 300 sampled points, and dL/dh
    against the oracle on all points."""
    rng = np.random.default_rng(906)
    wl = workloads.random_points(906, 2001, 5200.0, 10.0, 520, 540, 160.0, oracle.GAUSSIAN)
    G = rng.normal(0, 1, (540, 520)) + 0.5 * np.sin(np.arange(520) / 17.0)[None, :]
    gxy, gw, gh = kde.grid_backward(_dev(wl.xy, torch.float64), _dev(wl.w, torch.float32),
                                    wl.origin, wl.cell, 520, 540, wl.h, _dev(G, torch.float32))
    sel = np.sort(rng.choice(wl.n, 300, replace=False))
    rw, rxy, _ = oracle.kde_vjp_gauss(wl.xy, wl.w, wl.origin, wl.cell, 520, 540, wl.h, G,
                                      pts=sel)
    got_w, got_xy = gw.cpu().numpy()[sel], gxy.cpu().numpy()[sel]
    assert rel_linf(got_w, rw) <= TOL_GRAD
    assert rel_linf(got_xy, rxy) <= TOL_GRAD
    assert _rel_per_point(got_w, rw) <= 10 * TOL_GRAD
    _, _, rh = oracle.kde_vjp_gauss(wl.xy, wl.w, wl.origin, wl.cell, 520, 540, wl.h, G)
    assert gh == pytest.approx(rh, rel=TOL_GRAD)


def test_contraction_adjoint_zero_cotangent():
    wl, _ = _case(seed=907, n=129)
    G = np.zeros((wl.ny, wl.nx))
    gxy, gw, gh = kde.grid_backward(_dev(wl.xy, torch.float64), _dev(wl.w, torch.float32),
                                    wl.origin, wl.cell, wl.nx, wl.ny, wl.h,
                                    _dev(G, torch.float32), path="tc_split16")
    assert not gxy.any() and not gw.any() and gh == 0.0
