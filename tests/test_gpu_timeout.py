"""The bounded device-side waits give up with KDE_ETIMEOUT and leave the CUDA
context usable (a wait on a barrier nothing signals, and the bin sort's
look-back waiting for a chunk that never publishes; no fault, no trap)."""
import numpy as np
import pytest

import oracle
import workloads
from kde_testutil import TOL_SPLIT, rel_linf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2004_13653_gb300 as kde  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return kde.load(build_if_stale=True)


def test_wait_times_out_and_context_survives(lib):
    rc = lib.kde_diag_wait_timeout(200_000_000, None)  # 0.2 s
    assert rc == kde.KDE_ETIMEOUT
    assert "gave up" in lib.kde_last_error().decode()
    wl = workloads.config1()
    F = kde.grid(torch.as_tensor(wl.xy, device="cuda"), torch.as_tensor(wl.w, device="cuda"),
                 wl.origin, wl.cell, wl.nx, wl.ny, wl.h, "gaussian", flags=kde.FLAG_SYNC)
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, oracle.GAUSSIAN)
    assert rel_linf(F.cpu().numpy(), ref) <= TOL_SPLIT


def test_wait_limit_validated(lib):
    assert lib.kde_diag_wait_timeout(10, None) == kde.KDE_EINVAL
    assert lib.kde_diag_wait_timeout(10_000_000_000, None) == kde.KDE_EINVAL


def test_sort_lookback_times_out_and_context_survives(lib):
    rc = lib.kde_diag_sort_wait_timeout(100_000_000, None)  # 0.1 s
    assert rc == kde.KDE_ETIMEOUT
    assert "role 31" in lib.kde_last_error().decode()
    # the cutoff path (which runs the same sort) still matches the oracle
    wl = workloads.random_points(530, 2000, 900.0, 10.0, 97, 61, 30.0, oracle.EPANECHNIKOV)
    F = kde.grid(torch.as_tensor(wl.xy, device="cuda"), torch.as_tensor(wl.w, device="cuda"),
                 wl.origin, wl.cell, wl.nx, wl.ny, wl.h, "epanechnikov", path="cutoff",
                 flags=kde.FLAG_SYNC)
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, oracle.EPANECHNIKOV)
    assert rel_linf(F.cpu().numpy(), ref) <= 1e-6
    assert lib.kde_diag_sort_wait_timeout(10, None) == kde.KDE_EINVAL
