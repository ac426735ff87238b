"""GB300 (sm_103a) kernel density estimation of vessel positions on a grid.

Thin ctypes binding over the C ABI declared in ``include/kde.h``; it only
marshals arguments (torch tensors or numpy arrays, device or host) to the
library, whose kernels do every step of the computation.  There is no CPU
fallback: importing the binding on a machine where ``libkde_gb300.so`` is
missing raises.

Calls run on the torch current stream (or ``stream=``) and share the
library's device workspace, which only stream order protects: calls in
flight at the same time on different streams of one device each pass their
own ``workspace=`` (a device buffer of ``workspace_size(...)`` bytes).
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

KERNELS = {"uniform": 0, "triangular": 1, "epanechnikov": 2, "quartic": 3, "triweight": 4,
           "tricube": 5, "gaussian": 6, "cosine": 7}
RADIAL = 8  # radial variant of Table 1 kernel k: RADIAL + k ("radial_<name>")
KERNELS.update({"radial_" + k: RADIAL + v for k, v in list(KERNELS.items())})
PATHS = {"auto": 0, "simt": 1, "tc_fp16": 2, "tc_split16": 3, "cutoff": 4}
FLAG_SYNC, FLAG_SKIP_ZERO, FLAG_CTA_PAIR, FLAG_ONE_CTA = 1, 2, 4, 8
FLAG_LONLAT, FLAG_HOST_ASYNC = 16, 32

KDE_OK, KDE_EINVAL, KDE_ENOMEM, KDE_ECUDA, KDE_ETIMEOUT, KDE_ENOTSUP, KDE_EDATA = 0, -1, -2, -3, -4, -5, -6
_ERRNAMES = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "ENOTSUP", -6: "EDATA"}


class KDEError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"KDE_{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class KdeArgs(ctypes.Structure):
    _fields_ = [("points", ctypes.c_void_p), ("weights", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("origin_x", ctypes.c_double), ("origin_y", ctypes.c_double),
                ("cell", ctypes.c_double), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("h", ctypes.c_double), ("kernel_id", ctypes.c_int32), ("out", ctypes.c_void_p)]


class KdeOpts(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("flags", ctypes.c_uint32), ("stream", ctypes.c_void_p),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t),
                ("split_k", ctypes.c_int32), ("k_chunk", ctypes.c_int32),
                ("tile_n", ctypes.c_int32), ("max_ctas", ctypes.c_int32),
                ("timing_events", ctypes.c_void_p), ("stage_points", ctypes.c_int32),
                ("lat0_deg", ctypes.c_double)]


class KdeTiling(ctypes.Structure):
    _fields_ = [("tile_n", ctypes.c_int32), ("k_chunk", ctypes.c_int32),
                ("split_k", ctypes.c_int32), ("stage_points", ctypes.c_int32),
                ("flags", ctypes.c_uint32)]


EXPORTS = ("kde_default_opts", "kde_grid", "kde_grid_ex", "kde_workspace_size",
           "kde_project_mercator", "kde_grid_batched", "kde_grid_batched_tiled",
           "kde_grid_backward", "kde_lscv_grid",
           "kde_last_error", "kde_release", "kde_version", "kde_launch_count",
           "kde_diag_exclusive_scan", "kde_grid_noalloc", "kde_diag_wait_timeout",
           "kde_grid_binned", "kde_dp_simplify", "kde_diag_peak_rates",
           "kde_diag_sort_wait_timeout", "kde_set_stream")

_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_stale: bool = False) -> ctypes.CDLL:
    """Load libkde_gb300.so (building it first when asked).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_stale:
        _build.build()
    if not os.path.exists(_build.LIB_PATH):
        raise ImportError(f"{_build.LIB_PATH} is missing: build it with "
                          "`python -m paper_2004_13653_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(_build.LIB_PATH)
    P = ctypes.POINTER
    vp, i64, i32, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.kde_default_opts.argtypes = [P(KdeOpts)]
    lib.kde_default_opts.restype = None
    lib.kde_grid.argtypes = [vp, vp, i64, P(ctypes.c_double * 2), d, i32, i32, d, i32, vp]
    lib.kde_grid.restype = i32
    lib.kde_grid_ex.argtypes = [P(KdeArgs), P(KdeOpts)]
    lib.kde_grid_ex.restype = i32
    lib.kde_workspace_size.argtypes = [P(KdeArgs), P(KdeOpts), P(ctypes.c_size_t)]
    lib.kde_workspace_size.restype = i32
    lib.kde_project_mercator.argtypes = [vp, i64, d, vp, vp]
    lib.kde_project_mercator.restype = i32
    lib.kde_grid_batched.argtypes = [P(KdeArgs), i32, P(KdeOpts)]
    lib.kde_grid_batched.restype = i32
    lib.kde_grid_batched_tiled.argtypes = [P(KdeArgs), P(KdeTiling), i32, P(KdeOpts)]
    lib.kde_grid_batched_tiled.restype = i32
    lib.kde_grid_backward.argtypes = [P(KdeArgs), vp, vp, vp, P(ctypes.c_double), P(KdeOpts)]
    lib.kde_grid_backward.restype = i32
    lib.kde_lscv_grid.argtypes = [P(KdeArgs), vp, P(ctypes.c_double), vp, vp, vp,
                                  P(ctypes.c_double), P(KdeOpts)]
    lib.kde_lscv_grid.restype = i32
    lib.kde_last_error.argtypes = []
    lib.kde_last_error.restype = ctypes.c_char_p
    lib.kde_release.argtypes = []
    lib.kde_release.restype = i32
    lib.kde_launch_count.argtypes = []
    lib.kde_launch_count.restype = ctypes.c_int64
    lib.kde_grid_noalloc.argtypes = [vp, vp, i64, P(ctypes.c_double * 2), d, i32, i32, d, i32,
                                     vp, vp]
    lib.kde_grid_noalloc.restype = i32
    lib.kde_grid_binned.argtypes = [vp, vp, i64, i64, P(ctypes.c_double * 2), d, i32, i32, d, i32,
                                    i32, i32, vp, vp, P(ctypes.c_int64), P(KdeOpts)]
    lib.kde_grid_binned.restype = i32
    lib.kde_dp_simplify.argtypes = [vp, vp, i64, i64, d, vp, vp, vp, P(ctypes.c_int64),
                                    P(ctypes.c_int), P(KdeOpts)]
    lib.kde_dp_simplify.restype = i32
    lib.kde_diag_wait_timeout.argtypes = [i64, vp]
    lib.kde_diag_wait_timeout.restype = i32
    lib.kde_diag_sort_wait_timeout.argtypes = [i64, vp]
    lib.kde_diag_sort_wait_timeout.restype = i32
    lib.kde_set_stream.argtypes = [vp]
    lib.kde_set_stream.restype = None
    lib.kde_diag_peak_rates.argtypes = [P(ctypes.c_double * 3), vp]
    lib.kde_diag_peak_rates.restype = i32
    lib.kde_diag_exclusive_scan.argtypes = [vp, vp, i64, i32, vp]
    lib.kde_diag_exclusive_scan.restype = i32
    lib.kde_version.argtypes = []
    lib.kde_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def check(rc: int) -> None:
    if rc != KDE_OK:
        raise KDEError(rc, load().kde_last_error().decode())


# ------------------------------------------------------------- marshalling

def _ptr(t):
    """Raw address of a torch tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return t.data_ptr()
    if not t.flags["C_CONTIGUOUS"]:
        raise ValueError("arrays must be C-contiguous")
    return t.ctypes.data


def _count(t) -> int:
    return int(t.numel()) if hasattr(t, "numel") else int(t.size)


def _check_dtype(t, name, kinds):
    if t is None:
        return
    dt = str(t.dtype)
    if not any(k in dt for k in kinds):
        raise TypeError(f"{name} must be {kinds[0]}, got {dt}")


def kernel_id(kernel) -> int:
    return KERNELS[kernel] if isinstance(kernel, str) else int(kernel)


def make_args(points, weights, origin, cell, nx, ny, h, kernel, out) -> KdeArgs:
    _check_dtype(points, "points", ("float64",))
    _check_dtype(weights, "weights", ("float32",))
    _check_dtype(out, "out", ("float32",))
    n = _count(points) // 2 if points is not None else 0
    if weights is not None and _count(weights) != n:
        raise ValueError("weights must have one entry per point")
    if out is not None and _count(out) != int(nx) * int(ny):
        raise ValueError("out must have nx*ny elements")
    return KdeArgs(_ptr(points), _ptr(weights), n, float(origin[0]), float(origin[1]), float(cell),
                   int(nx), int(ny), float(h), kernel_id(kernel), _ptr(out))


def make_opts(path="auto", flags=0, stream=None, workspace=None, split_k=0, k_chunk=0,
              tile_n=0, max_ctas=0, timing_events=None, stage_points=0,
              lat0_deg=0.0) -> KdeOpts:
    o = KdeOpts()
    load().kde_default_opts(ctypes.byref(o))
    o.path = PATHS[path] if isinstance(path, str) else int(path)
    o.flags = int(flags)
    if stream is not None:
        o.stream = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    if workspace is not None:
        o.workspace = _ptr(workspace)
        o.workspace_bytes = _count(workspace) * workspace.element_size()
    o.split_k, o.k_chunk, o.tile_n, o.max_ctas = int(split_k), int(k_chunk), int(tile_n), int(max_ctas)
    o.stage_points = int(stage_points)
    o.lat0_deg = float(lat0_deg)
    if timing_events is not None:
        # keep the array alive as long as the options object
        o._events = timing_events
        o.timing_events = ctypes.cast(timing_events, ctypes.c_void_p)
    return o


def event_pair(start, end):
    """cudaEvent_t[2] from two recorded torch.cuda.Event objects."""
    return (ctypes.c_void_p * 2)(start.cuda_event, end.cuda_event)


def launch_count() -> int:
    return int(load().kde_launch_count())


def _current_stream(device):
    import torch
    return torch.cuda.current_stream(device)


# ------------------------------------------------------------------ the API

def grid(points, weights, origin, cell, nx, ny, h, kernel="gaussian", out=None, path="auto",
         flags=0, stream=None, **tiling):
    """Density on the nx x ny grid (kde_grid_ex).  See include/kde.h.

    points: [n,2] float64 metres (torch cuda/cpu tensor or numpy array), or
    (lon, lat) degrees with flags=FLAG_LONLAT and lat0_deg= the standard
    latitude; weights: [n] float32 or None; returns out ([ny, nx] float32),
    allocated like points when not given.  Runs on the torch current stream of
    the points' device unless `stream` is given; host buffers make it
    synchronous unless flags has FLAG_HOST_ASYNC.  Tiling keywords, workspace=,
    timing_events= and lat0_deg= go to kde_opts.
    """
    import torch
    if out is None:
        if isinstance(points, torch.Tensor):
            out = torch.empty((int(ny), int(nx)), dtype=torch.float32, device=points.device)
        else:
            import numpy as np
            out = np.empty((int(ny), int(nx)), dtype=np.float32)
    if stream is None and isinstance(out, torch.Tensor) and out.is_cuda:
        stream = _current_stream(out.device)
    a = make_args(points, weights, origin, cell, nx, ny, h, kernel, out)
    o = make_opts(path, flags, stream, **tiling)
    check(load().kde_grid_ex(ctypes.byref(a), ctypes.byref(o)))
    return out


def grid_simple(points, weights, origin, cell, nx, ny, h, kernel, out):
    """kde_grid: the plain entry point (the set_stream stream, legacy unless
    set; AUTO path; synchronous)."""
    a = make_args(points, weights, origin, cell, nx, ny, h, kernel, out)
    org = (ctypes.c_double * 2)(float(origin[0]), float(origin[1]))
    check(load().kde_grid(a.points, a.weights, a.n, ctypes.byref(org), a.cell, a.nx, a.ny, a.h,
                          a.kernel_id, a.out))
    return out


def set_stream(stream=None) -> None:
    """kde_set_stream: the stream grid_simple (kde_grid) runs on and waits for,
    for the calling thread; a torch.cuda.Stream, a raw cudaStream_t as int, or
    None for the legacy default stream."""
    if stream is None:
        ptr = None
    else:
        ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    load().kde_set_stream(ctypes.c_void_p(ptr))


def workspace_size(points, weights, origin, cell, nx, ny, h, kernel, out, **opts) -> int:
    a = make_args(points, weights, origin, cell, nx, ny, h, kernel, out)
    o = make_opts(**opts)
    b = ctypes.c_size_t(0)
    check(load().kde_workspace_size(ctypes.byref(a), ctypes.byref(o), ctypes.byref(b)))
    return int(b.value)


def grid_batched(instances, path="auto", flags=0, stream=None, tilings=None, **tiling):
    """kde_grid_batched: many densities, one persistent launch per path family.

    instances: sequence of dicts with keys points, weights, origin, cell, nx,
    ny, h, kernel and optionally out (device tensors).  tilings: optional
    sequence (one per instance) of dicts with keys of kde_tiling (tile_n,
    k_chunk, split_k, stage_points, flags) or None, e.g. from
    autotune.tune_batch; then kde_grid_batched_tiled runs the batch.  Returns
    the outputs.
    """
    import torch
    args = (KdeArgs * max(len(instances), 1))()
    outs = []
    for k, d in enumerate(instances):
        out = d.get("out")
        if out is None:
            out = torch.empty((int(d["ny"]), int(d["nx"])), dtype=torch.float32,
                              device=d["points"].device)
        outs.append(out)
        args[k] = make_args(d["points"], d.get("weights"), d["origin"], d["cell"], d["nx"],
                            d["ny"], d["h"], d.get("kernel", "gaussian"), out)
    if stream is None and outs:
        stream = _current_stream(outs[0].device)
    o = make_opts(path, flags, stream, **tiling)
    if tilings is None:
        check(load().kde_grid_batched(args, len(instances), ctypes.byref(o)))
        return outs
    if len(tilings) != len(instances):
        raise ValueError("one tiling per instance")
    tl = (KdeTiling * max(len(instances), 1))()
    for k, d in enumerate(tilings):
        for key, v in (d or {}).items():
            setattr(tl[k], key, int(v))
    check(load().kde_grid_batched_tiled(args, tl, len(instances), ctypes.byref(o)))
    return outs


def grid_backward(points, weights, origin, cell, nx, ny, h, grad_out, stream=None,
                  want_h=True, path="auto"):
    """kde_grid_backward (Gaussian): (dL/dpoints [n,2] f32, dL/dw [n] f32, dL/dh).
    path: "auto", "simt" (the window kernel) or "tc_split16" (the contractions)."""
    import torch
    n = _count(points) // 2
    gxy = torch.empty((n, 2), dtype=torch.float32, device=points.device)
    gw = torch.empty(n, dtype=torch.float32, device=points.device)
    gh = ctypes.c_double(0.0)
    if stream is None:
        stream = _current_stream(points.device)
    a = make_args(points, weights, origin, cell, nx, ny, h, "gaussian", grad_out)
    o = make_opts(path, 0, stream)
    check(load().kde_grid_backward(ctypes.byref(a), _ptr(grad_out.contiguous()), _ptr(gxy),
                                   _ptr(gw), ctypes.byref(gh) if want_h else None,
                                   ctypes.byref(o)))
    return gxy, gw, (gh.value if want_h else None)


def lscv_grid(F, points, weights, origin, cell, nx, ny, h, stream=None):
    """kde_lscv_grid (Gaussian): (loss, dL/dF, direct dL/dw, direct dL/dpoints, direct dL/dh)."""
    import torch
    n = _count(points) // 2
    G = torch.empty_like(F)
    gw = torch.empty(n, dtype=torch.float32, device=points.device)
    gxy = torch.empty((n, 2), dtype=torch.float32, device=points.device)
    loss = ctypes.c_double(0.0)
    gh = ctypes.c_double(0.0)
    if stream is None:
        stream = _current_stream(points.device)
    a = make_args(points, weights, origin, cell, nx, ny, h, "gaussian", F)
    o = make_opts("auto", 0, stream)
    check(load().kde_lscv_grid(ctypes.byref(a), _ptr(F), ctypes.byref(loss), _ptr(G), _ptr(gw),
                               _ptr(gxy), ctypes.byref(gh), ctypes.byref(o)))
    return loss.value, G, gw, gxy, gh.value


def grid_binned(points, offsets, origin, cell, nx, ny, h, kernel="gaussian", window=0,
                interpolate=True, stream=None, count=True):
    """kde_grid_binned: (density [ny,nx] f32, counts [ny,nx] int32, interpolated cells).
    With count=False the call stays asynchronous and the third value is None."""
    import torch
    dev = points.device
    out = torch.empty((int(ny), int(nx)), dtype=torch.float32, device=dev)
    counts = torch.empty((int(ny), int(nx)), dtype=torch.int32, device=dev)
    n = _count(points) // 2
    ntraj = 0 if offsets is None else _count(offsets) - 1
    org = (ctypes.c_double * 2)(float(origin[0]), float(origin[1]))
    added = ctypes.c_int64(0)
    if stream is None:
        stream = _current_stream(dev)
    o = make_opts("auto", 0, stream)
    check(load().kde_grid_binned(_ptr(points), _ptr(offsets), ntraj, n, ctypes.byref(org),
                                 float(cell), int(nx), int(ny), float(h), kernel_id(kernel),
                                 int(window), int(bool(interpolate)), _ptr(counts), _ptr(out),
                                 ctypes.byref(added) if count else None, ctypes.byref(o)))
    return out, counts, (int(added.value) if count else None)


def dp_simplify(points, offsets, eps, stream=None, compact=True):
    """kde_dp_simplify: (keep [n] uint8, kept points [n_kept, 2] float64 or None,
    their trajectory offsets [ntraj+1] int64 or None, iterations)."""
    import torch
    dev = points.device
    n = _count(points) // 2
    keep = torch.empty(n, dtype=torch.uint8, device=dev)
    ntraj = 1 if offsets is None else _count(offsets) - 1
    out = torch.empty((n, 2), dtype=torch.float64, device=dev) if compact else None
    out_off = torch.empty(ntraj + 1, dtype=torch.int64, device=dev) if compact else None
    kept = ctypes.c_int64(0)
    its = ctypes.c_int(0)
    if stream is None:
        stream = _current_stream(dev)
    o = make_opts("auto", 0, stream)
    check(load().kde_dp_simplify(_ptr(points), _ptr(offsets), ntraj, n, float(eps), _ptr(keep),
                                 _ptr(out), _ptr(out_off), ctypes.byref(kept), ctypes.byref(its),
                                 ctypes.byref(o)))
    if compact:
        out = out[:kept.value]
    return keep, out, out_off, its.value


def project_mercator(lonlat, lat0_deg, out=None, stream=None):
    """Eq. 1-4 on the device: [n,2] (lon, lat) degrees float64 -> metres."""
    import torch
    if out is None:
        out = torch.empty_like(lonlat)
    if stream is None:
        stream = _current_stream(lonlat.device)
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    check(load().kde_project_mercator(_ptr(lonlat), _count(lonlat) // 2, float(lat0_deg),
                                      _ptr(out), s))
    return out


def exclusive_scan(values, per_block=2048, out=None):
    """kde_diag_exclusive_scan on a uint32-compatible int32 cuda tensor."""
    import torch
    if out is None:
        out = torch.empty_like(values)
    check(load().kde_diag_exclusive_scan(_ptr(values), _ptr(out), _count(values), int(per_block),
                                         None))
    return out


def peak_rates(stream=None) -> dict:
    """kde_diag_peak_rates: the measured tcgen05 FP16 rates (TFLOP/s, CTA
    pairs and single CTAs) and the MUFU ex2 rate (1e12 per second)."""
    r = (ctypes.c_double * 3)()
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    check(load().kde_diag_peak_rates(ctypes.byref(r), stream))
    return {"mma_f16_pair_tflops": r[0], "mma_f16_cta_tflops": r[1], "ex2_tera_per_s": r[2]}


def release() -> None:
    check(load().kde_release())


def version() -> str:
    return load().kde_version().decode()
