"""Shared helpers for the parity tests: the error metric and cell sampling.

err = max_{c in S} |F_gpu(c) - F_oracle(c)| / max_{c in S} F_oracle(c), over a
set S of cells that contains the GPU argmax and its 8x8 neighbourhood.
"""
import numpy as np

TOL_FP32 = 1e-6     # FP32 SIMT path
TOL_FP16 = 2e-3     # single-FP16 tensor path
TOL_SPLIT = 1e-5    # split-FP16 tensor path
TOL_GRAD = 1e-4     # gradients (relative)


def rel_linf(gpu, ref):
    gpu = np.asarray(gpu, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    denom = np.max(np.abs(ref))
    assert denom > 0, "reference is identically zero"
    return float(np.max(np.abs(gpu - ref)) / denom)


def sample_cells(F_gpu, count=256, seed=0, neighbourhood=8):
    """Flat cell indices: GPU argmax + neighbourhood, the corners, random."""
    F = np.asarray(F_gpu)
    ny, nx = F.shape
    j0, i0 = np.unravel_index(int(np.argmax(F)), F.shape)
    cells = set()
    for dj in range(-neighbourhood // 2, neighbourhood // 2):
        for di in range(-neighbourhood // 2, neighbourhood // 2):
            j, i = j0 + dj, i0 + di
            if 0 <= j < ny and 0 <= i < nx:
                cells.add(j * nx + i)
    for j, i in ((0, 0), (0, nx - 1), (ny - 1, 0), (ny - 1, nx - 1)):
        cells.add(j * nx + i)
    rng = np.random.default_rng(seed)
    while len(cells) < count:
        cells.add(int(rng.integers(0, nx * ny)))
    return np.array(sorted(cells), dtype=np.int64)


def clear_of_support_edge(wl, radial, margin=1e-5):
    """The uniform kernel jumps at the edge of its support, and the GPU takes
    that decision in FP32 while the oracle takes it in FP64: a pair within
    rounding of the edge may count on one side only.  Returns the workload
    without the points that have a cell centre within `margin` (relative) of
    the edge (|s| = 1 or |t| = 1; |u| = 1 for the radial kernel)."""
    import dataclasses
    ox, oy = wl.origin
    x = wl.xy[:, 0]
    y = wl.xy[:, 1]
    i0 = np.floor((x - ox) / wl.cell - wl.h / wl.cell - 1).astype(np.int64)
    j0 = np.floor((y - oy) / wl.cell - wl.h / wl.cell - 1).astype(np.int64)
    span = int(np.ceil(2 * wl.h / wl.cell)) + 3
    di = np.arange(span)
    s = (ox + (i0[:, None] + di[None, :] + 0.5) * wl.cell - x[:, None]) / wl.h
    t = (oy + (j0[:, None] + di[None, :] + 0.5) * wl.cell - y[:, None]) / wl.h
    if radial:
        r = np.sqrt(s[:, :, None] ** 2 + t[:, None, :] ** 2)
        bad = np.any(np.abs(r - 1.0) < margin, axis=(1, 2))
    else:
        bad = np.any(np.abs(np.abs(s) - 1.0) < margin, axis=1) | \
            np.any(np.abs(np.abs(t) - 1.0) < margin, axis=1)
    keep = ~bad
    return dataclasses.replace(wl, local=wl.local[keep], w=wl.w[keep],
                               offsets=np.array([0, int(keep.sum())], dtype=np.int64))
