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
