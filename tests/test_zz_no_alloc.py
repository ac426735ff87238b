"""kde_grid_noalloc, the entry point for callers that cannot allocate device
memory (its scratch is a static device array), against the allocating entry
point kde_grid_ex on the same path, through the C ABI.

This file is collected last so that a run stopping at the first failure has
run every other test first; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from kde_testutil import TOL_FP32, rel_linf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2004_13653_gb300 as kde  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return kde.load(build_if_stale=True)


def _noalloc(lib, wl, kernel, out, stream):
    pts = torch.as_tensor(np.ascontiguousarray(wl.xy), dtype=torch.float64, device="cuda")
    w = torch.as_tensor(wl.w, dtype=torch.float32, device="cuda")
    org = (ctypes.c_double * 2)(*wl.origin)
    rc = lib.kde_grid_noalloc(pts.data_ptr(), w.data_ptr(), wl.n, ctypes.byref(org), wl.cell,
                              wl.nx, wl.ny, wl.h, kernel, out.data_ptr(), stream.cuda_stream)
    assert rc == kde.KDE_OK, lib.kde_last_error().decode()
    return pts, w


def test_noalloc_matches_allocating_entry_point_twice_in_a_row(lib):
    stream = torch.cuda.current_stream()
    cases = [(workloads.config1(), oracle.GAUSSIAN),
             (workloads.random_points(800, 700, 900.0, 7.5, 97, 61, 26.0, oracle.QUARTIC),
              oracle.QUARTIC)]
    for wl, kernel in cases:  # the second call reuses (and must not see) the first's scratch
        out = torch.full((wl.ny, wl.nx), np.nan, dtype=torch.float32, device="cuda")
        pts, w = _noalloc(lib, wl, kernel, out, stream)
        torch.cuda.synchronize()
        ref = kde.grid(pts, w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, kernel, path="simt",
                       flags=kde.FLAG_SYNC)
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert rel_linf(got, ref.cpu().numpy()) <= TOL_FP32


def test_noalloc_takes_no_device_memory(lib):
    # after one call (which loads the kernels and looks up the scratch), further
    # calls leave the device's free memory exactly as it was
    wl = workloads.config1()
    out = torch.empty((wl.ny, wl.nx), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    pts, w = _noalloc(lib, wl, oracle.GAUSSIAN, out, stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for kernel in (oracle.GAUSSIAN, 14):  # 14: the radial Gaussian, the same density
        org = (ctypes.c_double * 2)(*wl.origin)
        rc = lib.kde_grid_noalloc(pts.data_ptr(), w.data_ptr(), wl.n, ctypes.byref(org), wl.cell,
                                  wl.nx, wl.ny, wl.h, kernel, out.data_ptr(), stream.cuda_stream)
        assert rc == kde.KDE_OK, lib.kde_last_error().decode()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_in_a_captured_graph_matches_the_oracle(lib):
    """Captured into a CUDA graph in global capture mode (an allocation by any
    thread fails the capture), after one plain call that looks up the scratch:
    every replay gives the plain call's values bit for bit, within FP32 of the
    oracle."""
    wl = workloads.config1()
    pts = torch.as_tensor(np.ascontiguousarray(wl.xy), dtype=torch.float64, device="cuda")
    w = torch.as_tensor(wl.w, dtype=torch.float32, device="cuda")
    org = (ctypes.c_double * 2)(*wl.origin)

    def call(out):
        rc = lib.kde_grid_noalloc(pts.data_ptr(), w.data_ptr(), wl.n, ctypes.byref(org), wl.cell,
                                  wl.nx, wl.ny, wl.h, oracle.GAUSSIAN, out.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
        assert rc == kde.KDE_OK, lib.kde_last_error().decode()

    plain = torch.full((wl.ny, wl.nx), np.nan, dtype=torch.float32, device="cuda")
    call(plain)
    torch.cuda.synchronize()
    out = torch.full_like(plain, np.nan)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="global"):
        call(out)
    for _ in range(2):
        out.fill_(np.nan)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, plain)
    ref = oracle.kde_grid(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, oracle.GAUSSIAN)
    assert rel_linf(out.cpu().numpy(), ref) <= TOL_FP32


def test_noalloc_rejects_inputs_beyond_its_scratch(lib):
    wl = workloads.random_points(801, 1_000_000, 5000.0, 10.0, 64, 64, 30.0, oracle.GAUSSIAN)
    out = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    pts = torch.as_tensor(wl.xy, dtype=torch.float64, device="cuda")
    org = (ctypes.c_double * 2)(*wl.origin)
    rc = lib.kde_grid_noalloc(pts.data_ptr(), None, wl.n, ctypes.byref(org), wl.cell, 64, 64,
                              wl.h, oracle.GAUSSIAN, out.data_ptr(), None)
    assert rc == kde.KDE_EINVAL
    assert "static maximum" in lib.kde_last_error().decode()
