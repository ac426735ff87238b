"""FP64 CPU oracle for the KDE-on-grid hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path under
``paper_2004_13653_gb300/`` never imports it, and this package imports
nothing from there: the two share no code.

The arithmetic lives in ``kde_oracle.c`` (plain C, FP64, no tuning); this module
compiles it with gcc on first use and marshals numpy arrays through ctypes.
Every function cites the passage of arXiv 2004.13653 it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kde_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# kernel ids, in Table 1 order
UNIFORM, TRIANGULAR, EPANECHNIKOV, QUARTIC, TRIWEIGHT, TRICUBE, GAUSSIAN, COSINE = range(8)
KERNEL_NAMES = ("uniform", "triangular", "epanechnikov", "quartic", "triweight",
                "tricube", "gaussian", "cosine")

# WGS84 ellipsoid (reading: the paper names a and e but gives no values)
WGS84_A = 6378137.0
WGS84_E2 = 0.00669437999014


def build(force: bool = False) -> str:
    """Compile kde_oracle.c into liboracle.so (gcc, -O2, IEEE semantics)."""
    with _lock:
        stale = (not os.path.exists(_LIB_PATH)
                 or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
        if force or stale:
            tmp = _LIB_PATH + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                                   "-pthread", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
        vp = ctypes.c_void_p
        lib.oracle_kernel_1d.argtypes = [i32, d]
        lib.oracle_kernel_1d.restype = d
        lib.oracle_kernel_radial.argtypes = [i32, d]
        lib.oracle_kernel_radial.restype = d
        lib.oracle_mercator.argtypes = [vp, i64, d, d, d, vp]
        lib.oracle_mercator.restype = None
        lib.oracle_kde_cells.argtypes = [vp, vp, i64, d, d, d, i32, i32, d, i32,
                                         vp, i64, vp, i32]
        lib.oracle_kde_cells.restype = i32
        lib.oracle_kde_vjp_gauss.argtypes = [vp, vp, i64, d, d, d, i32, i32, d,
                                             vp, vp, i64, vp, vp, vp, i32]
        lib.oracle_kde_vjp_gauss.restype = i32
        lib.oracle_lscv_loss.argtypes = [vp, vp, vp, i64, d, d, d, i32, i32, d]
        lib.oracle_lscv_loss.restype = d
        lib.oracle_lscv_cotangent.argtypes = [vp, vp, vp, i64, d, d, d, i32, i32, vp]
        lib.oracle_lscv_cotangent.restype = None
        lib.oracle_ved.argtypes = [d] * 6
        lib.oracle_ved.restype = d
        lib.oracle_dp.argtypes = [vp, vp, i64, d, vp]
        lib.oracle_dp.restype = i32
        lib.oracle_count_matrix.argtypes = [vp, vp, i64, d, d, d, i32, i32, i32, vp]
        lib.oracle_count_matrix.restype = i64
        lib.oracle_convolve.argtypes = [vp, i32, i32, d, d, i32, i32, i64, vp]
        lib.oracle_convolve.restype = None
        _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    return None if a is None else a.ctypes.data


RADIAL = 8  # kernel id of the radial variant of Table 1 kernel k: RADIAL + k


def kernel_radial(kid: int, r) -> np.ndarray:
    """K(r): the radial variant of Table 1 kernel kid (0..7) on the unit disk,
    normalised over the plane."""
    lib = _load()
    r = np.asarray(r, dtype=np.float64)
    out = np.array([lib.oracle_kernel_radial(int(kid), float(v)) for v in r.ravel()])
    return out.reshape(r.shape)


def kernel_1d(kid: int, s) -> np.ndarray:
    """k(s): one factor of the product kernel f(s,t) = k(s) k(t) (Table 1)."""
    lib = _load()
    s = np.asarray(s, dtype=np.float64)
    out = np.array([lib.oracle_kernel_1d(int(kid), float(v)) for v in s.ravel()])
    return out.reshape(s.shape)


def mercator(lonlat_deg, lat0_deg: float, a: float = WGS84_A,
             e2: float = WGS84_E2) -> np.ndarray:
    """Eq. 1-4: (lon, lat) degrees, interleaved [n,2] -> (x, y) metres [n,2]."""
    lib = _load()
    ll = _f64(lonlat_deg).reshape(-1, 2)
    out = np.empty_like(ll)
    lib.oracle_mercator(_ptr(ll), ll.shape[0], float(lat0_deg), float(a), float(e2), _ptr(out))
    return out


def kde_cells(xy, w, origin, cell, nx, ny, h, kid, cells=None, threads=0) -> np.ndarray:
    """Eq. 7 read as the direct sum, Table 1 kernels, at cell centres.

    xy: [n,2] absolute metres; w: [n] weights or None (unit); origin: (ox, oy)
    lower-left corner of cell (0,0); cells: flat indices j*nx+i, or None for
    the whole grid (returned as [ny, nx]).
    """
    lib = _load()
    xy = _f64(xy).reshape(-1, 2)
    n = xy.shape[0]
    wv = None if w is None else _f64(w).reshape(-1)
    if wv is not None and wv.shape[0] != n:
        raise ValueError("weights length mismatch")
    if cells is None:
        ncells = int(nx) * int(ny)
        cv = None
    else:
        cv = np.ascontiguousarray(np.asarray(cells, dtype=np.int64).reshape(-1))
        ncells = cv.shape[0]
    out = np.empty(ncells, dtype=np.float64)
    rc = lib.oracle_kde_cells(_ptr(xy), _ptr(wv), n, float(origin[0]), float(origin[1]),
                              float(cell), int(nx), int(ny), float(h), int(kid),
                              _ptr(cv), ncells, _ptr(out), int(threads))
    if rc != 0:
        raise ValueError(f"oracle_kde_cells rejected its arguments (rc={rc})")
    return out.reshape(int(ny), int(nx)) if cells is None else out


def kde_grid(xy, w, origin, cell, nx, ny, h, kid, threads=0) -> np.ndarray:
    """The whole grid, shape [ny, nx] (row j = y index, column i = x index)."""
    return kde_cells(xy, w, origin, cell, nx, ny, h, kid, None, threads)


def kde_vjp_gauss(xy, w, origin, cell, nx, ny, h, G, pts=None, threads=0):
    """Gradient of L = sum_ij G_ij F_ij for the Gaussian kernel.

    Returns (dL/dw [m], dL/dxy [m,2], dL/dh or None) for the listed points
    (all points when pts is None; dL/dh only then).
    """
    lib = _load()
    xy = _f64(xy).reshape(-1, 2)
    n = xy.shape[0]
    wv = None if w is None else _f64(w).reshape(-1)
    Gv = _f64(G).reshape(-1)
    if Gv.shape[0] != int(nx) * int(ny):
        raise ValueError("cotangent shape mismatch")
    pv = None if pts is None else np.ascontiguousarray(np.asarray(pts, dtype=np.int64))
    m = n if pv is None else pv.shape[0]
    gw = np.empty(m)
    gxy = np.empty((m, 2))
    gh = np.zeros(1)
    rc = lib.oracle_kde_vjp_gauss(_ptr(xy), _ptr(wv), n, float(origin[0]), float(origin[1]),
                                  float(cell), int(nx), int(ny), float(h), _ptr(Gv), _ptr(pv),
                                  m, _ptr(gw), _ptr(gxy), _ptr(gh), int(threads))
    if rc != 0:
        raise ValueError(f"oracle_kde_vjp_gauss failed (rc={rc})")
    return gw, gxy, (float(gh[0]) if pv is None else None)


def lscv_loss(F, xy, w, origin, cell, nx, ny, h) -> float:
    """Grid LSCV loss (Gaussian); F is the [ny,nx] density from kde_grid."""
    lib = _load()
    Fv = _f64(F).reshape(-1)
    xy = _f64(xy).reshape(-1, 2)
    wv = None if w is None else _f64(w).reshape(-1)
    return lib.oracle_lscv_loss(_ptr(Fv), _ptr(xy), _ptr(wv), xy.shape[0], float(origin[0]),
                                float(origin[1]), float(cell), int(nx), int(ny), float(h))


def lscv_cotangent(F, xy, w, origin, cell, nx, ny) -> np.ndarray:
    """dL/dF of the grid LSCV loss, shape [ny, nx]."""
    lib = _load()
    Fv = _f64(F).reshape(-1)
    xy = _f64(xy).reshape(-1, 2)
    wv = None if w is None else _f64(w).reshape(-1)
    G = np.empty_like(Fv)
    lib.oracle_lscv_cotangent(_ptr(Fv), _ptr(xy), _ptr(wv), xy.shape[0], float(origin[0]),
                              float(origin[1]), float(cell), int(nx), int(ny), _ptr(G))
    return G.reshape(int(ny), int(nx))


def lscv_value_and_grad(xy, w, origin, cell, nx, ny, h, threads=0):
    """LSCV loss and its gradient w.r.t. (w, xy, h), all FP64.

    The gradient is the chain rule through F (the VJP above with the LSCV
    cotangent) plus the loss's direct dependence on w_p, x_p and h.
    """
    xy = _f64(xy).reshape(-1, 2)
    n = xy.shape[0]
    wv = np.ones(n) if w is None else _f64(w).reshape(-1)
    F = kde_grid(xy, wv, origin, cell, nx, ny, h, GAUSSIAN, threads)
    L = lscv_loss(F, xy, wv, origin, cell, nx, ny, h)
    G = lscv_cotangent(F, xy, wv, origin, cell, nx, ny)
    gw, gxy, gh = kde_vjp_gauss(xy, wv, origin, cell, nx, ny, h, G, None, threads)
    # direct terms of -(2/N) sum_p w_p bilerp(F - F_p, x_p): through the
    # bilinear weights (x_p), the weight w_p (twice: the factor and F_p) and
    # F_p's own dependence on x_p and h; F_p(g) = w_p S(g), S = exp(-r^2/2h^2)/(2 pi N h^2)
    ox, oy = float(origin[0]), float(origin[1])
    for p in range(n):
        fx = (xy[p, 0] - ox) / cell - 0.5
        fy = (xy[p, 1] - oy) / cell - 0.5
        i0, j0 = int(np.floor(fx)), int(np.floor(fy))
        ax, ay = fx - i0, fy - j0
        v = s = dvx = dvy = dsx = dsy = sh = 0.0
        for b in (0, 1):
            for a in (0, 1):
                ii, jj = i0 + a, j0 + b
                if ii < 0 or jj < 0 or ii >= nx or jj >= ny:
                    continue
                dx = ox + (ii + 0.5) * cell - xy[p, 0]
                dy = oy + (jj + 0.5) * cell - xy[p, 1]
                r2 = dx * dx + dy * dy
                S = np.exp(-0.5 * r2 / (h * h)) / (2.0 * np.pi * n * h * h)
                f = F[jj, ii]
                wx = ax if a else 1.0 - ax
                wy = ay if b else 1.0 - ay
                ex = (1.0 if a else -1.0) / cell * wy  # d(wx wy)/dx_p
                ey = (1.0 if b else -1.0) / cell * wx
                v += wx * wy * f
                s += wx * wy * S
                dvx += ex * f
                dvy += ey * f
                dsx += ex * S + wx * wy * S * dx / (h * h)
                dsy += ey * S + wx * wy * S * dy / (h * h)
                sh += wx * wy * S * (r2 / h ** 3 - 2.0 / h)
        gw[p] += -2.0 / n * (v - 2.0 * wv[p] * s)
        gxy[p, 0] += -2.0 / n * wv[p] * (dvx - wv[p] * dsx)
        gxy[p, 1] += -2.0 / n * wv[p] * (dvy - wv[p] * dsy)
        gh += 2.0 / n * wv[p] * wv[p] * sh
    return L, gw, gxy, gh


def ved(p, s, e) -> float:
    """Eq. 9: distance from p to the line through s and e."""
    return _load().oracle_ved(float(p[0]), float(p[1]), float(s[0]), float(s[1]),
                              float(e[0]), float(e[1]))


def douglas_peucker(xy, offsets, eps: float) -> np.ndarray:
    """Sec. III-B: boolean keep-mask over the concatenated trajectories."""
    lib = _load()
    xy = _f64(xy).reshape(-1, 2)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    keep = np.zeros(xy.shape[0], dtype=np.uint8)
    rc = lib.oracle_dp(_ptr(xy), _ptr(off), off.shape[0] - 1, float(eps), _ptr(keep))
    if rc != 0:
        raise MemoryError("oracle_dp failed")
    return keep.astype(bool)


def count_matrix(xy, offsets, origin, cell, nx, ny, interpolate=True):
    """Sec. IV-B / Algorithm 3: int32 count matrix [ny, nx] of the fixes, with the
    Eq. InterX/InterY interpolation of skipped cells; returns (counts, added)."""
    lib = _load()
    xy = _f64(xy).reshape(-1, 2)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    counts = np.zeros(int(nx) * int(ny), dtype=np.int32)
    added = lib.oracle_count_matrix(_ptr(xy), _ptr(off), off.shape[0] - 1, float(origin[0]),
                                    float(origin[1]), float(cell), int(nx), int(ny),
                                    int(bool(interpolate)), _ptr(counts))
    return counts.reshape(int(ny), int(nx)), int(added)


def convolve(counts, cell, h, kid, window, n_points) -> np.ndarray:
    """Eq. 7: the window x window stencil f(s,t) = k(s cell/h) k(t cell/h)/(N h^2)."""
    lib = _load()
    c = np.ascontiguousarray(np.asarray(counts, dtype=np.int32))
    ny, nx = c.shape
    out = np.empty((ny, nx), dtype=np.float64)
    lib.oracle_convolve(_ptr(c), int(nx), int(ny), float(cell), float(h), int(kid), int(window),
                        int(n_points), _ptr(out))
    return out
