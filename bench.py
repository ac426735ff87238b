#!/usr/bin/env python
"""Throughput of the KDE-on-grid hot path on GB300.

Workload: 20M AIS-like points (40,000 synthetic trajectories: 70% lane traffic,
20% port clusters, 10% uniform) over a 100 km box, 4096 x 4096 grid of
24.4140625 m cells, Gaussian kernel, h = 100 m.  One step = one kde_grid_ex
call on the (lon, lat) inputs: Mercator projection (FP64) fused with the
centring / hi-lo split -> density on the tensor cores (split-FP16 by default)
-> split-K reduce.

Metric: point.cell evaluations per second (N * nx * ny per step), in
Gpoint.cell/s, for the whole job.  Inputs are resident in HBM when the timed
region starts (they exceed the 129 MB L2: 320 MB of lon/lat), and `e2e`
repeats the step through the same call with pinned host buffers: the library
copies the inputs in and the grid out on the call's stream inside the timed
region (asynchronous host mode, two streams and two workspaces so one step's
copies overlap the other's kernels).  `--impl reference` times the FP64 CPU
oracle instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "KDE Gpoint·cell/s, 20M pts×4096² grid: split-FP16 tensor vs FP32 at ≤1e-5 err"

# DRAM bytes (read + write) per launch of the contraction kernel on the default workload, from
# one ncu capture (profiles/k_tc_pair_dram_20M_4096sq.md); reported only while the kernel's
# sources hash to the value they had when the counters were taken.
TRAFFIC = {("tc_split16", 4096, 40_000): {
    "sources": ["paper_2004_13653_gb300/csrc/kde_tc2.cu", "paper_2004_13653_gb300/csrc/tc_ptx.cuh"],
    "sha256": "db07cca8451ff248c21dca5576e9915dc9c831ec5beae7bfa6b2a8e19bd9e100",
    "bytes": 1255729152 + 527909888}}


def sparse_products(xy, origin, cell, nx, ny, h):
    """Point-tile pairs the block-sparse contraction multiplies out: for each
    256 x 256 tile, the points of the 32 x 32-cell bins within 6.45 h sqrt(2 ln 2)
    of it (the library's binning, in FP64 here).  Times 65536 cells and 2 FLOP
    per product this is the contraction's algorithmic work."""
    import numpy as np
    sigma = 1.0 / (h * 1.17741002251547469101)
    cs = cell * sigma
    # the library's ranges widen the reach by the FP32 rounding margin of its bin keys
    reach = 6.45 + 1e-6 + 8.0 * 2.0 ** -24 * (max(nx, ny) * cs + 6.45)
    inv_binw = 1.0 / (32 * cs)
    nbx, nby = (nx + 31) // 32, (ny + 31) // 32
    X = (xy[:, 0] - origin[0]) * sigma
    Y = (xy[:, 1] - origin[1]) * sigma
    keep = (X >= -reach) & (Y >= -reach) & (X <= nx * cs + reach) & (Y <= ny * cs + reach)
    bx = np.clip(np.floor(X[keep] * inv_binw), 0, nbx - 1).astype(np.int64)
    by = np.clip(np.floor(Y[keep] * inv_binw), 0, nby - 1).astype(np.int64)
    H = np.bincount(by * nbx + bx, minlength=nbx * nby).reshape(nby, nbx)
    S = np.zeros((nby + 1, nbx + 1), np.int64)
    S[1:, 1:] = H.cumsum(0).cumsum(1)
    total = 0
    for tn in range((ny + 255) // 256):
        y0, y1 = (tn * 256 + 0.5) * cs - reach, (tn * 256 + 255.5) * cs + reach
        ly, hy = max(0, int(np.floor(y0 * inv_binw))), min(nby - 1, int(np.floor(y1 * inv_binw)))
        for tm in range((nx + 255) // 256):
            x0, x1 = (tm * 256 + 0.5) * cs - reach, (tm * 256 + 255.5) * cs + reach
            lx = max(0, int(np.floor(x0 * inv_binw)))
            hx = min(nbx - 1, int(np.floor(x1 * inv_binw)))
            total += S[hy + 1, hx + 1] - S[ly, hx + 1] - S[hy + 1, lx] + S[ly, lx]
    return int(total)


def cutoff_pairs(xy, origin, cell, nx, ny, h):
    """Point-cell pairs the cutoff path evaluates: every 16 x 16-cell output
    block reads the points of the sort bins (4, 8 or 16 cells, chosen from
    h/cell) whose points can lie within a bandwidth of its cell centres (the
    library's binning, in FP64 here)."""
    import numpy as np
    rc = h / cell
    S = 4 if rc <= 6.0 else 8 if rc <= 16.0 else 16
    while S < 64 and ((nx + S - 1) // S) * ((ny + S - 1) // S) > (1 << 24):
        S *= 2
    B, cs = 16, cell / h
    reach = 1.0 + 1e-6 + 8.0 * 2.0 ** -24 * (max(nx, ny) * cs + 1.0)  # as the library's ranges
    inv_binw = 1.0 / (S * cs)
    nbx, nby = (nx + S - 1) // S, (ny + S - 1) // S
    X = (xy[:, 0] - origin[0]) / h
    Y = (xy[:, 1] - origin[1]) / h
    keep = (X >= -1) & (Y >= -1) & (X <= nx * cs + 1) & (Y <= ny * cs + 1)
    bx = np.clip(np.floor(X[keep] * inv_binw), 0, nbx - 1).astype(np.int64)
    by = np.clip(np.floor(Y[keep] * inv_binw), 0, nby - 1).astype(np.int64)
    H = np.bincount(by * nbx + bx, minlength=nbx * nby).reshape(nby, nbx)
    C = np.zeros((nby + 1, nbx + 1), np.int64)
    C[1:, 1:] = H.cumsum(0).cumsum(1)

    def lo_hi(c0, n):
        lo = np.clip(np.floor(((c0 + 0.5) * cs - reach) * inv_binw), 0, n).astype(np.int64)
        hi = np.minimum(np.floor(((c0 + B - 0.5) * cs + reach) * inv_binw), n - 1).astype(np.int64)
        return lo, hi
    lx, hx = lo_hi(np.arange(0, nx, B), nbx)
    ly, hy = lo_hi(np.arange(0, ny, B), nby)
    LY, LX = np.meshgrid(ly, lx, indexing="ij")
    HY, HX = np.meshgrid(hy, hx, indexing="ij")
    ok = (LX <= HX) & (LY <= HY)
    HX1, HY1 = np.where(ok, HX + 1, 0), np.where(ok, HY + 1, 0)
    LX, LY = np.where(ok, LX, 0), np.where(ok, LY, 0)
    reach_pts = C[HY1, HX1] - C[LY, HX1] - C[HY1, LX] + C[LY, LX]
    return int(B * B * reach_pts.sum())


def support_pairs(xy, origin, cell, nx, ny, h):
    """Point-cell pairs inside the square support |s| <= 1, |t| <= 1 of the
    product kernels (offsets in bandwidths): the algorithmic work of the
    cutoff path, sum over points of (cells per row) x (cells per column)."""
    import numpy as np
    X = (np.asarray(xy[:, 0], np.float64) - origin[0]) / cell
    Y = (np.asarray(xy[:, 1], np.float64) - origin[1]) / cell
    r = h / cell

    def span(c, n):
        # cell centres i + 1/2 within r of c, for i in [0, n)
        lo = np.maximum(np.ceil(c - r - 0.5), 0.0)
        hi = np.minimum(np.floor(c + r - 0.5), n - 1.0)
        return np.maximum(hi - lo + 1.0, 0.0)
    return int((span(X, nx) * span(Y, ny)).sum())


def cutoff_roofline(pairs, support, kernel_ms, n, nx, ny, peaks, peak_pairs):
    """The cutoff path's two rooflines: evaluated pairs against the FP32 ALU
    peak (the binding one), and its algorithmic bytes (the points read by the
    centring and by the sort's passes and the gather, about 60 B per point, and
    the grid written once) against the measured HBM rate; plus the pairs inside
    the supports, the work the method itself defines."""
    sec = kernel_ms * 1e-3
    gbs = (60.0 * n + 4.0 * nx * ny) / sec / 1e9
    return {"bound": "alu", "achieved": pairs / sec / 1e12, "peak": peak_pairs / 1e12,
            "unit": "Tpair/s", "frac": pairs / sec / peak_pairs, "traffic": None,
            "support_pairs": support, "support_tpair_s": support / sec / 1e12,
            "hbm": {"achieved_gbs": gbs, "peak_gbs": peaks["hbm_gbs"],
                    "frac": gbs / peaks["hbm_gbs"]}}


def measured_traffic(path, grid, points):
    import hashlib
    t = TRAFFIC.get((path, grid, points))
    if not t:
        return None
    h = hashlib.sha256()
    for f in t["sources"]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return t["bytes"] if h.hexdigest() == t["sha256"] else None
UNIT = "Gpoint·cell/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--path", default="tc_split16",
                    choices=["tc_split16", "tc_fp16", "simt", "cutoff"])
    ap.add_argument("--kernel", default="gaussian",
                    help="Table 1 kernel (the cutoff path needs a compact one)")
    ap.add_argument("--flags", type=int, default=0, help="extra KDE_FLAG_* bits")
    ap.add_argument("--extra", action="store_true",
                    help="also measure the batched, cutoff and LSCV workloads (slower)")
    ap.add_argument("--grid", type=int, default=4096, help="grid side (default: the 4096^2 workload)")
    ap.add_argument("--points", type=int, default=40_000, help="trajectories of 500 fixes")
    ap.add_argument("--simt-grid", type=int, default=4096,
                    help="grid side for the FP32 SIMT comparison (same points; 0 = skip)")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-instance batch leg")
    ap.add_argument("--no-configs12", action="store_true",
                    help="skip the legs of the 2,000-fix and 1M-fix workloads")
    ap.add_argument("--no-lscv", action="store_true", help="skip the LSCV bandwidth-fit leg")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint leg")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="run only the adjoint leg (window kernel vs contractions)")
    ap.add_argument("--adjoint-traj", type=int, default=2000,
                    help="trajectories of 500 fixes for the adjoint leg (default 1M fixes)")
    ap.add_argument("--adjoint-h-m", type=float, default=800.0,
                    help="bandwidth of the adjoint leg in metres (16.4 cells)")
    ap.add_argument("--no-peak-probe", action="store_true",
                    help="skip the measured tensor-core and ex2 rates")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sparse", action="store_true", help="skip the block-sparse leg")
    ap.add_argument("--cpu-cells", type=int, default=1200)
    ap.add_argument("--split-k", type=int, default=0)
    ap.add_argument("--k-chunk", type=int, default=0)
    ap.add_argument("--tile-n", type=int, default=0)
    ap.add_argument("--h-m", type=float, default=0.0,
                    help="bandwidth in metres (default: the workload's 100 m)")
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    elif torch.cuda.is_available():
        torch.cuda.set_device(local)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value):
    """The slowest rank's time (every rank ran the same replica workload)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world, evals, ms):
    """Whole-job rate of N replicas (weak scaling): every rank evaluated `evals`
    point-cell pairs, the job took the slowest rank's `ms`."""
    return world * evals / (ms * 1e-3) / 1e9


def make_workload(args):
    import workloads
    wl = workloads.config3(n_traj=args.points, grid=args.grid)
    if args.h_m > 0:
        wl.h = args.h_m
    ll, corner, lat0 = wl.lonlat()
    return wl, ll, corner, lat0


def run_ours(args):
    import numpy as np
    import torch

    import paper_2004_13653_gb300 as kde

    world, rank, local = dist_setup(args)
    if args.adjoint_only:
        kde.load(build_if_stale=True)
        if rank == 0:
            print(json.dumps({"adjoint": adjoint_leg(torch.device("cuda", local), args, local)}))
        return
    dev = torch.device("cuda", local)
    kde.load(build_if_stale=True)
    peaks, peak_kind = load_peaks()

    wl, ll, corner, lat0 = make_workload(args)
    n, nx, ny = wl.n, wl.nx, wl.ny
    lonlat_dev = torch.as_tensor(ll, dtype=torch.float64, device=dev)
    w_dev = torch.as_tensor(wl.w, dtype=torch.float32, device=dev)
    out_dev = torch.empty((ny, nx), dtype=torch.float32, device=dev)
    corner_dev = torch.tensor([corner], dtype=torch.float64, device=dev)
    origin = kde.project_mercator(corner_dev, lat0).cpu().numpy()[0]
    # projected fixes for the host-side work counts and the oracle (not timed)
    xy_dev = kde.project_mercator(lonlat_dev, lat0)
    stream = torch.cuda.current_stream(dev)
    tiling = dict(split_k=args.split_k, k_chunk=args.k_chunk, tile_n=args.tile_n)

    def step(events=None, path=args.path, out=out_dev, gx=nx, gy=ny, flags=args.flags):
        # one call: Eq. 1-4 fused into the centring, then the density
        kde.grid(lonlat_dev, w_dev, origin, wl.cell, gx, gy, wl.h, args.kernel, out=out,
                 path=path, flags=flags | kde.FLAG_LONLAT, lat0_deg=lat0, stream=stream,
                 timing_events=events, **tiling)

    def new_pair():
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        b.record(stream)
        return a, b

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    pairs = [new_pair() for _ in range(args.steps)]
    torch.cuda.synchronize()

    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    launches0 = kde.launch_count()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        step(kde.event_pair(*pairs[k]))
    t1.record(stream)
    torch.cuda.synchronize()
    launches = kde.launch_count() - launches0
    barrier(world)
    clk = clocks.stop()
    ms = t0.elapsed_time(t1) / args.steps
    ms = max_over_ranks(world, ms)
    kernel_ms = statistics.mean(a.elapsed_time(b) for a, b in pairs)
    evals = float(n) * nx * ny
    value = replica_value(world, evals, ms)

    # roofline of the dominant kernel
    if args.path in ("simt", "cutoff"):
        # per pair one FMA; per 32-point batch and 128 x 64-cell CTA the factors
        # are tabulated once, 6144 evaluations of ~6 FP32 ops (3 FADD, FMUL,
        # weight FMUL; MUFU aside), 0.14 ops per pair -> 1.14 FP32 ops per pair
        # (the cutoff path is charged the same per evaluated pair)
        clk_hz = peaks.get("sm_max_mhz", 2070.0) * 1e6
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak_pairs = alu_peak_pairs(peaks, sms)
        pairs = evals
        if args.path == "cutoff":  # only the pairs of the bins within reach are evaluated
            pairs = cutoff_pairs(xy_dev.cpu().numpy().reshape(-1, 2), origin, wl.cell, nx, ny,
                                 wl.h)
        achieved = pairs / (kernel_ms * 1e-3)
        roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_pairs / 1e12,
                "unit": "Tpair/s", "frac": achieved / peak_pairs, "traffic": None,
                "peak_source": f"FP32 issue 128/clk/SM at {clk_hz/1e6:.0f} MHz"}
        if args.path == "cutoff":
            xy_np = xy_dev.cpu().numpy().reshape(-1, 2)
            roof = dict(cutoff_roofline(pairs, support_pairs(xy_np, origin, wl.cell, nx, ny, wl.h),
                                        kernel_ms, n, nx, ny, peaks, peak_pairs),
                        peak_source=roof["peak_source"])
    else:
        products = 3 if args.path == "tc_split16" else 1
        flops = 2.0 * products * evals
        if args.flags & kde.FLAG_SKIP_ZERO:  # only the pairs within reach are multiplied
            xy_proj = xy_dev.cpu().numpy().reshape(-1, 2)  # the projected fixes
            flops = 2.0 * products * 65536.0 * sparse_products(xy_proj, origin, wl.cell, nx, ny,
                                                                wl.h)
        peak = peaks["bf16_tflops_sustained"]
        achieved = flops / (kernel_ms * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": measured_traffic(args.path, args.grid, args.points) if not args.flags
                else None,
                "peak_source": f"{peak_kind} bf16 sustained (FP16 dense rate taken equal)"}

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"tc_split16": "f16x2(hi/lo)->f32", "tc_fp16": "f16->f32",
                  "simt": "f32", "cutoff": "f32"}[args.path] + ", f64 projection/centring",
        "data": "synthetic",
        "config": {"workload": f"{n} AIS-like pts, {nx}x{ny} grid, cell {wl.cell} m, "
                               f"h={wl.h} m, {args.kernel}",
                   "path": args.path, "points": n, "grid": [nx, ny], "h_m": wl.h,
                   "l2": "inputs (320 MB lon/lat + 80 MB weights) larger than L2",
                   "parallelism": f"replicas x{world}"},
        "kernel_ms": kernel_ms,
        "roofline": roof,
        "gpu_launches": int(launches),
        "clocks": clk,
    }

    simt_out = None
    if rank == 0 and args.path not in ("simt", "cutoff") and args.simt_grid > 0:
        # the FP32 SIMT path on the same fixes: one warm-up call on a small grid
        # (the kernel is the same at every grid size), then one timed step on
        # the stated grid
        sg = args.simt_grid
        small = torch.empty((512, 512), dtype=torch.float32, device=dev)
        step(path="simt", out=small, gx=512, gy=512)
        simt_out = torch.empty((sg, sg), dtype=torch.float32, device=dev)
        torch.cuda.synchronize()
        a, b = new_pair()
        simt_clocks = ClockSampler(local)
        simt_clocks.start()
        time.sleep(0.3)
        a.record(stream)
        step(path="simt", out=simt_out, gx=sg, gy=sg)
        b.record(stream)
        torch.cuda.synchronize()
        simt_ms = a.elapsed_time(b)
        simt = float(n) * sg * sg / (simt_ms * 1e-3) / 1e9
        result["simt_fp32"] = {"value": simt, "unit": UNIT, "grid": [sg, sg], "ms_per_step": simt_ms,
                               "steps": 1, "clocks": simt_clocks.stop(),
                               "note": "FP32 SIMT path, same fixes, one timed step (after a "
                                       "warm-up call on a 512^2 grid)"}
        result["tensor_vs_simt"] = value / world / simt
        if sg != nx:
            simt_out = None

    sparse_e2e = None  # the block-sparse step through the host-buffer call
    if not args.no_e2e:
        # End to end through the same call with host buffers: pinned (lon, lat)
        # and weights in, the pinned grid out; the library copies them on the
        # call's stream.  FLAG_HOST_ASYNC lets a call return once queued, so
        # steps alternate between two streams (each with its own workspace and
        # output buffer) and one step's copies overlap the other's kernels.
        lonlat_host = torch.empty(tuple(lonlat_dev.shape), dtype=torch.float64, pin_memory=True)
        lonlat_host.copy_(torch.as_tensor(ll))
        w_host = torch.empty(n, dtype=torch.float32, pin_memory=True)
        w_host.copy_(torch.as_tensor(wl.w))
        outs_host = [torch.empty((ny, nx), dtype=torch.float32, pin_memory=True) for _ in range(2)]
        flags_e2e = args.flags | kde.FLAG_LONLAT | kde.FLAG_HOST_ASYNC
        wsb = kde.workspace_size(lonlat_host, w_host, origin, wl.cell, nx, ny, wl.h, args.kernel,
                                 outs_host[0], path=args.path, flags=flags_e2e,
                                 lat0_deg=lat0, **tiling)
        ws = [torch.empty(wsb, dtype=torch.uint8, device=dev) for _ in range(2)]
        streams = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]

        def e2e_step(k, events=None):
            b = k % 2
            kde.grid(lonlat_host, w_host, origin, wl.cell, nx, ny, wl.h, args.kernel,
                     out=outs_host[b], path=args.path, flags=flags_e2e, lat0_deg=lat0,
                     stream=streams[b], workspace=ws[b], timing_events=events, **tiling)

        torch.cuda.synchronize()
        for k in range(2):
            e2e_step(k)
        torch.cuda.synchronize()
        e2e_pairs = [new_pair() for _ in range(args.steps)]
        torch.cuda.synchronize()
        barrier(world)
        e2e_clocks = ClockSampler(local)
        e2e_clocks.start()
        time.sleep(0.3)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(streams[0])
        streams[1].wait_event(e0)
        for k in range(args.steps):
            e2e_step(k, kde.event_pair(*e2e_pairs[k]))
        streams[0].wait_stream(streams[1])
        e1.record(streams[0])
        torch.cuda.synchronize()
        barrier(world)
        ems = max_over_ranks(world, e0.elapsed_time(e1) / args.steps)
        h2d_bytes = int(lonlat_host.numel() * 8 + w_host.numel() * 4)
        result["e2e"] = {"value": replica_value(world, evals, ems), "unit": UNIT,
                         "ms_per_step": ems,
                         "h2d_bytes_per_step": h2d_bytes,
                         "d2h_bytes_per_step": int(outs_host[0].numel() * 4),
                         "copies": "inside kde_grid_ex: host (lon, lat) and weights in, grid out, "
                                   "on the call's stream (KDE_FLAG_HOST_ASYNC; two streams, two "
                                   "workspaces)",
                         # the dominant kernel's own time inside this loop
                         "kernel_ms": statistics.mean(a.elapsed_time(b) for a, b in e2e_pairs),
                         "clocks": e2e_clocks.stop()}
        del ws
        if rank == 0 and args.path in ("tc_split16", "tc_fp16") and not args.flags \
                and not args.no_sparse:
            # the block-sparse step through the same host-buffer call: its
            # kernels take a hundredth of the dense step's, so the copies show
            flags_sp = flags_e2e | kde.FLAG_SKIP_ZERO
            wss = kde.workspace_size(lonlat_host, w_host, origin, wl.cell, nx, ny, wl.h,
                                     args.kernel, outs_host[0], path=args.path, flags=flags_sp,
                                     lat0_deg=lat0, **tiling)
            ws_sp = [torch.empty(wss, dtype=torch.uint8, device=dev) for _ in range(2)]

            def sp_step(k):
                b = k % 2
                kde.grid(lonlat_host, w_host, origin, wl.cell, nx, ny, wl.h, args.kernel,
                         out=outs_host[b], path=args.path, flags=flags_sp, lat0_deg=lat0,
                         stream=streams[b], workspace=ws_sp[b], **tiling)

            for k in range(4):
                sp_step(k)
            torch.cuda.synchronize()
            reps = 20
            e0.record(streams[0])
            streams[1].wait_event(e0)
            for k in range(reps):
                sp_step(k)
            streams[0].wait_stream(streams[1])
            e1.record(streams[0])
            torch.cuda.synchronize()
            sms_e2e = e0.elapsed_time(e1) / reps
            sparse_e2e = {"value": evals / (sms_e2e * 1e-3) / 1e9, "unit": UNIT,
                          "ms_per_step": sms_e2e, "h2d_bytes_per_step": h2d_bytes,
                          "d2h_bytes_per_step": int(outs_host[0].numel() * 4),
                          # input bytes per step over the step time: the copy rate the
                          # step sustains while they overlap the other stream's kernels
                          "h2d_gbs_at_step_rate": h2d_bytes / (sms_e2e * 1e-3) / 1e9,
                          "copies": result["e2e"]["copies"]}
            del ws_sp

    if rank == 0 and not args.no_peak_probe:
        # the tcgen05 FP16 and ex2 rates measured by the library's own probes,
        # at the clock the GPU runs at now (after the steps above)
        probe_clocks = ClockSampler(local)
        probe_clocks.start()
        time.sleep(0.2)
        rates = kde.peak_rates()
        result["measured_rates"] = dict(rates, clocks=probe_clocks.stop(),
                                        note="kde_diag_peak_rates: MMAs on resident operands, "
                                             "every SM, second of two passes")
        if roof["bound"] == "tensor":
            one_cta = args.flags & kde.FLAG_ONE_CTA  # CTA pairs are the default
            probe = rates["mma_f16_cta_tflops" if one_cta else "mma_f16_pair_tflops"]
            roof["frac_of_probe"] = roof["achieved"] / probe

    sample = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"], sample = cpu_baseline(args, wl, origin, ll, lat0, out_dev)
        if simt_out is not None and "simt_fp32" in result:
            import numpy as np
            cells, ref = sample
            Fs = simt_out.cpu().numpy().reshape(-1)[cells]
            result["simt_fp32"]["rel_linf_vs_oracle_on_sample"] = float(
                np.max(np.abs(Fs - ref)) / np.max(np.abs(ref)))
    del simt_out

    if rank == 0 and args.path in ("tc_split16", "tc_fp16") and not args.flags \
            and not args.no_sparse:
        result["block_sparse"] = sparse_leg(step, stream, out_dev, new_pair, kernel_ms, evals,
                                            sample)
        if sparse_e2e is not None:
            result["block_sparse"]["e2e"] = sparse_e2e
        products = 3 if args.path == "tc_split16" else 1
        pt = sparse_products(xy_dev.cpu().numpy().reshape(-1, 2), origin, wl.cell, nx, ny, wl.h)
        flops = 2.0 * products * 65536.0 * pt
        ach = flops / (result["block_sparse"]["kernel_ms"] * 1e-3) / 1e12
        peak = peaks["bf16_tflops_sustained"]
        result["block_sparse"]["point_tile_pairs"] = pt
        result["block_sparse"]["roofline"] = {
            "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak, "traffic": None,
            "note": "FLOPs of the products within reach over the whole sparse step (sort, "
                    "work list, contraction, reduce)"}

    if rank == 0 and args.extra:
        result["binned_estimator"] = binned_leg(dev, wl, xy_dev, origin, out_dev)
    if rank == 0 and not (args.no_batched and args.no_lscv and args.no_adjoint and
                          args.no_configs12 and not args.extra):
        del lonlat_dev, xy_dev, out_dev
        torch.cuda.empty_cache()
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        if not args.no_configs12:
            result["configs12"] = configs12_leg(dev, peaks, sms, local)
        if not args.no_batched:
            result["batched"] = batched_leg(dev, peaks, sms, local)
        if not args.no_lscv:
            result["lscv_fit"] = lscv_leg(dev, local)
        if not args.no_adjoint:
            result["adjoint"] = adjoint_leg(dev, args, local)
        if args.extra:
            result["extra"] = extra_workloads(dev)

    if rank == 0:
        print(json.dumps(result))


def _time(fn, reps=3):
    import torch
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def extra_workloads(dev):
    """The other rows of the hot path on their own workloads: the binned
    cutoff path (1M lane points, 1024^2, Epanechnikov), the GPU
    Douglas-Peucker on the 2M raw lane fixes (eps = 10 m), and one forward,
    adjoint and LSCV evaluation on its output (1024^2, h = 150 m)."""
    import numpy as np
    import torch

    import paper_2004_13653_gb300 as kde
    import workloads
    out = {}
    wl = workloads.config2(kernel=2)
    pts = torch.as_tensor(wl.xy, dtype=torch.float64, device=dev)
    w = torch.as_tensor(wl.w, device=dev)
    F = torch.empty((wl.ny, wl.nx), device=dev)
    ms = _time(lambda: kde.grid(pts, w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h, "epanechnikov",
                                out=F, path="cutoff"))
    out["cutoff_epanechnikov_1M_1024sq"] = {
        "ms": ms, "Gpoint_cell_per_s": wl.n * wl.nx * wl.ny / ms / 1e6,
        "note": "definition-level rate (N nx ny / time); the path evaluates only the support"}
    ms = _time(lambda: kde.grid(pts, w, wl.origin, wl.cell, wl.nx, wl.ny, wl.h,
                                "radial_epanechnikov", out=F))
    out["cutoff_radial_epanechnikov_1M_1024sq"] = {
        "ms": ms, "Gpoint_cell_per_s": wl.n * wl.nx * wl.ny / ms / 1e6,
        "note": "the radial variant K(|u|) on the unit disk, same points and grid"}
    raw = workloads.config5_raw()
    xy = torch.as_tensor(raw.xy, dtype=torch.float64, device=dev)
    off = torch.as_tensor(raw.offsets, device=dev)
    dp_ms = _time(lambda: kde.dp_simplify(xy, off, 10.0), reps=3)
    keep, thin, _, its = kde.dp_simplify(xy, off, 10.0)
    # each kept fix stands for the raw fixes up to the next kept one
    idx = np.flatnonzero(keep.cpu().numpy())
    rep = np.diff(np.append(idx, raw.n)).astype(np.float32)
    out["douglas_peucker_2M_eps10m"] = {
        "points": int(raw.n), "kept": int(idx.size), "iterations": its, "ms": dp_ms,
        "Mpoint_per_s": raw.n / dp_ms / 1e3}
    w0 = torch.as_tensor(rep, device=dev)
    # one forward, one adjoint (dL/dpoints, dL/dw, dL/dh for a random cotangent)
    # and one grid-LSCV evaluation on the thinned fixes, h = 150 m
    G = torch.rand((raw.ny, raw.nx), device=dev, generator=torch.Generator(dev).manual_seed(5))
    args5 = (thin, w0, raw.origin, raw.cell, raw.nx, raw.ny, 150.0)
    fwd_ms = _time(lambda: kde.grid(*args5, "gaussian"), reps=5)
    fwd_sparse_ms = _time(lambda: kde.grid(*args5, "gaussian", flags=kde.FLAG_SKIP_ZERO), reps=5)
    bwd_ms = _time(lambda: kde.grid_backward(*args5, G), reps=5)
    F5 = kde.grid(*args5, "gaussian")
    lscv_ms = _time(lambda: kde.lscv_grid(F5, *args5), reps=5)
    out["forward_adjoint_lscv_1024sq"] = {
        "points": int(thin.shape[0]), "forward_ms": fwd_ms,
        "forward_block_sparse_ms": fwd_sparse_ms, "adjoint_ms": bwd_ms, "lscv_ms": lscv_ms,
        "note": "adjoint: a warp per 32 points, each over its +-8h window in turn "
                "(dL/dw, dL/dpoints, dL/dh)"}
    return out


def alu_peak_pairs(peaks, sms):
    """ALU roofline of the SIMT and cutoff paths in pair evaluations per second:
    1.14 FP32 instructions per pair (one FMA plus the factor tabulation) at
    128 FP32 lanes per SM per clock."""
    clk_hz = peaks.get("sm_max_mhz", 2070.0) * 1e6
    return sms * clk_hz * min(128 / 1.14, 16 / (6144 / (32 * 8192)))


def configs12_leg(dev, peaks, sms, local):
    """Configs 1 and 2 on their own: the 2,000-fix Gaussian on 64^2 through the
    FP32 SIMT path against the oracle on every cell, and the 1M lane fixes on
    1024^2 (h = 150 m) with the Gaussian on the FP32 SIMT path and on the
    split-FP16 tensor path and the Epanechnikov on the cutoff path, each timed
    as a whole call (device-resident inputs; centring, sort and reduce
    included) and checked on sampled cells."""
    import numpy as np
    import torch

    import oracle
    import paper_2004_13653_gb300 as kde
    import workloads
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from kde_testutil import sample_cells

    def err(F, ref):
        return float(np.max(np.abs(F - ref)) / np.max(np.abs(ref)))

    out = {}
    c1 = workloads.config1()
    xy1 = torch.as_tensor(c1.xy, dtype=torch.float64, device=dev)
    run1 = lambda: kde.grid(xy1, None, c1.origin, c1.cell, c1.nx, c1.ny, c1.h, "gaussian",
                            path="simt")
    ms1 = _time(run1, reps=20)
    ref1 = oracle.kde_grid(c1.xy, c1.w, c1.origin, c1.cell, c1.nx, c1.ny, c1.h, oracle.GAUSSIAN)
    out["config1_simt_fp32"] = {"points": c1.n, "grid": [c1.nx, c1.ny], "ms_per_call": ms1,
                                "rel_linf_vs_oracle_all_cells": err(run1().cpu().numpy(), ref1)}
    c2 = workloads.config2()
    xy2 = torch.as_tensor(c2.xy, dtype=torch.float64, device=dev)
    evals = float(c2.n) * c2.nx * c2.ny
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.2)
    res = {}
    for name, kernel, path, reps in (("gaussian_simt_fp32", "gaussian", "simt", 2),
                                     ("gaussian_tc_split16", "gaussian", "tc_split16", 5),
                                     ("epanechnikov_cutoff", "epanechnikov", "cutoff", 20)):
        call = lambda: kde.grid(xy2, None, c2.origin, c2.cell, c2.nx, c2.ny, c2.h, kernel,
                                path=path)
        res[name] = (_time(call, reps=reps), call().cpu().numpy())
    clk = clocks.stop()
    for kid, names in ((oracle.GAUSSIAN, ("gaussian_simt_fp32", "gaussian_tc_split16")),
                       (oracle.EPANECHNIKOV, ("epanechnikov_cutoff",))):
        cells = sample_cells(res[names[-1]][1], 256, seed=12)
        ref = oracle.kde_cells(c2.xy, c2.w, c2.origin, c2.cell, c2.nx, c2.ny, c2.h, kid, cells,
                               threads=os.cpu_count() or 1)
        for name in names:
            ms, F = res[name]
            out[f"config2_{name}"] = {"ms_per_call": ms, "value": evals / ms / 1e6, "unit": UNIT,
                                      "rel_linf_vs_oracle_on_sample":
                                          err(F.reshape(-1)[cells], ref)}
    tc = out["config2_gaussian_tc_split16"]
    tflops = 6.0 * evals / (tc["ms_per_call"] * 1e-3) / 1e12
    tc["roofline"] = {"bound": "tensor", "achieved": tflops,
                      "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s",
                      "frac": tflops / peaks["bf16_tflops_sustained"],
                      "note": "whole call: centring, contraction and split-K reduce"}
    tc["vs_simt"] = out["config2_gaussian_simt_fp32"]["ms_per_call"] / tc["ms_per_call"]
    cut = out["config2_epanechnikov_cutoff"]
    pairs = cutoff_pairs(c2.xy, c2.origin, c2.cell, c2.nx, c2.ny, c2.h)
    peak_a = alu_peak_pairs(peaks, sms)
    cut["roofline"] = dict(cutoff_roofline(pairs, support_pairs(c2.xy, c2.origin, c2.cell, c2.nx,
                                                                c2.ny, c2.h),
                                           cut["ms_per_call"], c2.n, c2.nx, c2.ny, peaks, peak_a),
                           note="evaluated pairs (16x16-cell blocks x points of the sort bins "
                                "within reach) over the whole call")
    out["config2_points"] = c2.n
    out["clocks"] = clk
    del xy1, xy2
    torch.cuda.empty_cache()
    return out


def batched_leg(dev, peaks, sms, local):
    """The 256-instance batch (point counts log-uniform 1e4..2e6, grid sides
    2^7..2^11, h in 50..800 m, Gaussian and Epanechnikov half and half) in one
    kde_grid_batched call, captured in a CUDA graph and replayed; parity on
    sampled cells of a few instances of each kernel; roofline = the time the
    instances would take at their own rooflines (tensor peak for the Gaussian
    contractions, ALU peak for the cutoff pairs) over the measured time."""
    import numpy as np
    import torch

    import oracle
    import paper_2004_13653_gb300 as kde
    import workloads
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from kde_testutil import sample_cells
    inst = workloads.config4_instances()
    insts = [dict(points=torch.as_tensor(x.xy, dtype=torch.float64, device=dev),
                  weights=torch.as_tensor(x.w, device=dev), origin=x.origin, cell=x.cell,
                  nx=x.nx, ny=x.ny, h=x.h, kernel=x.kernel) for x in inst]
    outs = [torch.empty((x.ny, x.nx), device=dev) for x in inst]
    for d, o in zip(insts, outs):
        d["out"] = o
    from paper_2004_13653_gb300 import autotune
    ms_default = _time(lambda: kde.grid_batched(insts), reps=2)
    # tiles per instance class from the autotuner (timed here on first use,
    # then cached), one persistent launch per tile family
    import tempfile
    t0 = time.perf_counter()
    tilings = autotune.tune_batch(insts, cache_path=os.path.join(tempfile.gettempdir(),
                                                                 "kde_bench_autotune.json"))
    tune_s = time.perf_counter() - t0
    ms = _time(lambda: kde.grid_batched(insts, tilings=tilings), reps=2)
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            kde.grid_batched(insts, stream=st, tilings=tilings)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    gms = _time(g.replay, reps=3)
    clk = clocks.stop()
    chosen = {}
    for t in tilings:
        if t is not None:
            k = ("pair" if t["flags"] == autotune.PAIR else "one-cta") + \
                f" {256 if t['flags'] == autotune.PAIR else 128}x{t['tile_n']} s{t['stage_points']}"
            chosen[k] = chosen.get(k, 0) + 1
    # parity: the largest instances of each kernel, 64 sampled cells each
    errs = {}
    for kid, name in ((6, "gaussian"), (2, "epanechnikov")):
        idx = sorted((k for k, x in enumerate(inst) if x.kernel == kid),
                     key=lambda k: -inst[k].n)[:3]
        worst = 0.0
        for k in idx:
            x = inst[k]
            F = outs[k].cpu().numpy()
            cells = sample_cells(F, 64, seed=k)
            ref = oracle.kde_cells(x.xy, x.w, x.origin, x.cell, x.nx, x.ny, x.h, x.kernel, cells,
                                   threads=os.cpu_count() or 1)
            worst = max(worst, float(np.max(np.abs(F.reshape(-1)[cells] - ref)) /
                                     np.max(np.abs(ref))))
        errs[name] = {"instances": idx, "rel_linf_vs_oracle_on_sample": worst}
    t_roof = 0.0
    peak_t = peaks["bf16_tflops_sustained"] * 1e12
    peak_a = alu_peak_pairs(peaks, sms)
    for x in inst:
        if x.kernel == 6:
            t_roof += 6.0 * x.n * x.nx * x.ny / peak_t
        else:
            t_roof += cutoff_pairs(x.xy, x.origin, x.cell, x.nx, x.ny, x.h) / peak_a
    pairs = float(sum(x.n * x.nx * x.ny for x in inst))
    del insts, outs, g
    torch.cuda.empty_cache()
    return {"instances": len(inst), "points": int(sum(x.n for x in inst)), "ms": ms,
            "graph_replay_ms": gms, "value": pairs / gms / 1e6, "unit": UNIT,
            "autotuned": {"tilings": chosen, "tuning_s": tune_s,
                          "ms_with_default_tiles": ms_default},
            "kernels": {"gaussian": sum(x.kernel == 6 for x in inst),
                        "epanechnikov": sum(x.kernel == 2 for x in inst)},
            "roofline": {"bound": "tensor+alu", "roofline_ms": t_roof * 1e3,
                         "frac": t_roof * 1e3 / gms,
                         "note": "sum over instances of work / peak (tensor: measured sustained "
                                 "bf16 for the split-FP16 contractions; ALU: FP32 issue for the "
                                 "evaluated cutoff pairs) over the measured replay time"},
            "parity": errs, "clocks": clk}


def lscv_leg(dev, local):
    """Config 5: the 2M raw lane fixes thinned by the GPU Douglas-Peucker at
    eps = 10 m, then 200 Adam steps of the grid LSCV loss over (log h, weight
    logits) on 1024^2 (forward, adjoint and loss kernels every step)."""
    import numpy as np
    import torch

    import oracle
    import paper_2004_13653_gb300 as kde
    import workloads
    from paper_2004_13653_gb300 import autograd as kag
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from kde_testutil import sample_cells
    raw = workloads.config5_raw()
    xy = torch.as_tensor(raw.xy, dtype=torch.float64, device=dev)
    off = torch.as_tensor(raw.offsets, device=dev)
    keep, thin, _, its = kde.dp_simplify(xy, off, 10.0)
    idx = np.flatnonzero(keep.cpu().numpy())
    rep = np.diff(np.append(idx, raw.n)).astype(np.float32)
    w0 = torch.as_tensor(rep, device=dev)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h, w, losses = kag.fit_bandwidth(thin, w0, raw.origin, raw.cell, raw.nx, raw.ny, 150.0,
                                     steps=200, lr=0.05)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    clk = clocks.stop()
    # parity at the fitted bandwidth: the density on sampled cells, and the
    # loss of the GPU grid recomputed by the oracle's loss function
    F = kde.grid(thin, w, raw.origin, raw.cell, raw.nx, raw.ny, h, "gaussian",
                 flags=kde.FLAG_SYNC)
    Fh = F.cpu().numpy()
    xyh = thin.cpu().numpy()
    wh = w.cpu().numpy().astype(np.float64)
    cells = sample_cells(Fh, 64, seed=9)
    ref = oracle.kde_cells(xyh, wh, raw.origin, raw.cell, raw.nx, raw.ny, h, oracle.GAUSSIAN, cells,
                           threads=os.cpu_count() or 1)
    loss_gpu = kde.lscv_grid(F, thin, w, raw.origin, raw.cell, raw.nx, raw.ny, h)[0]
    loss_or = oracle.lscv_loss(Fh, xyh, wh, raw.origin, raw.cell, raw.nx, raw.ny, h)
    return {"raw_points": int(raw.n), "points": int(thin.shape[0]), "dp_iterations": its,
            "steps": 200, "seconds": secs, "ms_per_step": secs * 1e3 / 200, "h0_m": 150.0,
            "h_final_m": h, "loss_first": losses[0], "loss_last": losses[-1],
            "parity": {"density_rel_linf_vs_oracle_on_sample":
                       float(np.max(np.abs(Fh.reshape(-1)[cells] - ref)) / np.max(np.abs(ref))),
                       "loss_rel_vs_oracle_same_grid": abs(loss_gpu - loss_or) / abs(loss_or)},
            "clocks": clk,
            "input": "GPU Douglas-Peucker output at eps = 10 m, initial weights = raw fixes each "
                     "kept fix stands for"}


def adjoint_leg(dev, args, local):
    """The adjoint (kde_grid_backward: dL/dw, dL/dpoints, dL/dh) of the config-2
    fixes on 1024^2 for a random cotangent at a wide bandwidth (default 800 m,
    16.4 cells): the +-8h window kernel and the two tensor-core contractions,
    both forced, timed, and checked against the oracle's VJP on sampled points.
    Roofline of the contractions: 2 x 3 x N_pad x nx_pad x ny_pad FP16
    multiply-adds against the measured sustained peak."""
    import numpy as np
    import torch

    import oracle
    import paper_2004_13653_gb300 as kde
    import workloads
    wl = workloads.config2(n_traj=args.adjoint_traj)
    h = args.adjoint_h_m
    pts = torch.as_tensor(wl.xy, dtype=torch.float64, device=dev)
    w = torch.as_tensor(wl.w, device=dev)
    G = torch.randn((wl.ny, wl.nx), device=dev, generator=torch.Generator(dev).manual_seed(11))
    res = {"points": int(wl.n), "grid": [wl.nx, wl.ny], "h_m": h, "h_cells": h / wl.cell}
    outs = {}
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    for path in ("simt", "tc_split16"):
        run = lambda: kde.grid_backward(pts, w, wl.origin, wl.cell, wl.nx, wl.ny, h, G,
                                        want_h=False, path=path)
        res[{"simt": "window_ms", "tc_split16": "contractions_ms"}[path]] = _time(run, reps=3)
        outs[path] = run()
    res["clocks"] = clocks.stop()
    rng = np.random.default_rng(12)
    sel = np.sort(rng.choice(wl.n, 128, replace=False))
    rw, rxy, _ = oracle.kde_vjp_gauss(wl.xy, wl.w, wl.origin, wl.cell, wl.nx, wl.ny, h,
                                      G.cpu().numpy().astype(np.float64), pts=sel,
                                      threads=os.cpu_count() or 1)
    for path, (gxy, gw, _) in outs.items():
        e_w = float(np.max(np.abs(gw.cpu().numpy()[sel] - rw)) / np.max(np.abs(rw)))
        e_xy = float(np.max(np.abs(gxy.cpu().numpy()[sel] - rxy)) / np.max(np.abs(rxy)))
        res[{"simt": "window", "tc_split16": "contractions"}[path] + "_rel_linf_vs_oracle"] = \
            max(e_w, e_xy)
    n_pad = (wl.n + 511) // 512 * 512
    pad = lambda v: (v + 255) // 256 * 256
    flops = 2 * 3 * 2.0 * n_pad * pad(wl.nx) * pad(wl.ny)
    peaks, _ = load_peaks()
    ach = flops / (res["contractions_ms"] * 1e-3) / 1e12
    res["roofline"] = {"bound": "tensor", "achieved": ach, "peak": peaks["bf16_tflops_sustained"],
                       "unit": "TFLOP/s", "frac": ach / peaks["bf16_tflops_sustained"],
                       "note": "both contractions and the cotangent tiling, whole call"}
    res["speedup"] = res["window_ms"] / res["contractions_ms"]
    return res


def sparse_leg(step, stream, out_dense, new_pair, dense_kernel_ms, evals, sample):
    """The same step with block-sparse skipping (KDE_FLAG_SKIP_ZERO): points
    sorted into bins, each tile reading only the bins within ~7.6 h, where
    every FP16 operand is exactly zero.  Same products, fewer of them; the
    rate is definition-level (N nx ny / time)."""
    import numpy as np
    import torch

    import paper_2004_13653_gb300 as kde
    out = torch.empty_like(out_dense)
    for _ in range(3):
        step(out=out, flags=kde.FLAG_SKIP_ZERO)
    torch.cuda.synchronize()
    reps = 10
    pairs = [new_pair() for _ in range(reps)]
    t0, t1 = new_pair()
    t0.record(stream)
    for k in range(reps):
        step(kde.event_pair(*pairs[k]), out=out, flags=kde.FLAG_SKIP_ZERO)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / reps
    kms = statistics.mean(a.elapsed_time(b) for a, b in pairs)
    res = {"ms_per_step": ms, "kernel_ms": kms, "value": evals / (ms * 1e-3) / 1e9, "unit": UNIT,
           "kernel_speedup_vs_dense": dense_kernel_ms / kms,
           "rel_linf_vs_dense": float((out - out_dense).abs().max() / out_dense.abs().max())}
    if sample is not None:
        cells, ref = sample
        F = out.cpu().numpy().reshape(-1)[cells]
        res["rel_linf_vs_oracle_on_sample"] = float(np.max(np.abs(F - ref)) / np.max(np.abs(ref)))
    res["note"] = ("kernel_ms covers the bin sort, the work list, the contraction and the "
                   "piece reduce; the skipped operands are exactly zero in FP16")
    return res


def binned_leg(dev, wl, xy_dev, origin, F_direct):
    """The paper's own estimator (Sec. IV-B: count matrix, interpolation of
    skipped cells, Eq. 7 convolution with a +-4h window) on the same fixes and
    grid, timed with and without interpolation; its difference from the direct
    sum (the headline path's output) is the binning error."""
    import torch

    import numpy as np

    import paper_2004_13653_gb300 as kde
    # only the lane vessels are tracks: the port-cluster and background fixes
    # are independent draws, so each is a trajectory of its own (interpolating
    # between them would draw segments no vessel sailed)
    fixes = int(wl.offsets[1] - wl.offsets[0])
    n_lane = int(round(0.7 * (len(wl.offsets) - 1))) * fixes
    offs = np.concatenate([wl.offsets[wl.offsets <= n_lane],
                           np.arange(n_lane + 1, wl.n + 1, dtype=np.int64)])
    off = torch.as_tensor(offs, device=dev)
    res = {"trajectories": int(len(offs) - 1)}
    for interp in (False, True):
        def call():
            return kde.grid_binned(xy_dev, off, origin, wl.cell, wl.nx, wl.ny, wl.h, "gaussian",
                                   0, interp, count=False)
        ms = _time(call, reps=5)
        F, _, added = kde.grid_binned(xy_dev, off, origin, wl.cell, wl.nx, wl.ny, wl.h,
                                      "gaussian", 0, interp)
        err = float((F - F_direct).abs().max() / F_direct.abs().max())
        res["interpolated" if interp else "plain"] = {
            "ms": ms, "Gpoint_cell_per_s": wl.n * wl.nx * wl.ny / ms / 1e6,
            "interpolated_cells": added, "rel_linf_vs_direct_sum": err}
    res["window"] = 2 * math.ceil(4 * wl.h / wl.cell) + 1
    res["note"] = ("definition-level rate (N nx ny / time); the estimator bins the fixes, "
                   "so it is an approximation of the direct sum")
    return res


def cpu_baseline(args, wl, origin, ll, lat0, out_dev):
    """The FP64 oracle on a bounded sample of cells of the same workload, on all
    host cores; also reports the GPU result's error on those cells."""
    import numpy as np

    import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from kde_testutil import sample_cells

    cores = os.cpu_count() or 1
    F = out_dev.cpu().numpy()
    cells = sample_cells(F, args.cpu_cells, seed=3)
    xy = oracle.mercator(ll, lat0)
    t = time.perf_counter()
    ref = oracle.kde_cells(xy, wl.w, origin, wl.cell, wl.nx, wl.ny, wl.h, oracle.GAUSSIAN, cells,
                           threads=cores)
    dt = time.perf_counter() - t
    err = float(np.max(np.abs(F.reshape(-1)[cells] - ref)) / np.max(np.abs(ref)))
    return {"value": len(cells) * wl.n / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(cells)} cells (GPU argmax 8x8 neighbourhood, corners, random) x "
                      f"all {wl.n} points, FP64, {dt:.1f} s",
            # the sample's time scaled to every cell of the grid (not measured)
            "extrapolated_full_grid_s": dt * wl.nx * wl.ny / len(cells),
            "gpu_err_rel_linf_on_sample": err}, (cells, ref)


def run_reference(args):
    """The FP64 CPU oracle as the reference arm: each step is a bounded sample
    (cells x all points) of the same workload, rank 0 only."""
    import numpy as np

    import oracle
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    wl, ll, corner, lat0 = make_workload(args)
    xy = oracle.mercator(ll, lat0)
    origin = oracle.mercator([corner], lat0)[0]
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(7)
    per_step = 24
    times = []
    for k in range(args.warmup + args.steps):
        cells = rng.choice(wl.nx * wl.ny, per_step, replace=False)
        t = time.perf_counter()
        oracle.kde_cells(xy, wl.w, origin, wl.cell, wl.nx, wl.ny, wl.h, oracle.GAUSSIAN, cells,
                         threads=cores)
        if k >= args.warmup:
            times.append(time.perf_counter() - t)
    step_s = sum(times) / len(times)
    value = per_step * wl.n / step_s / 1e9
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{wl.n} AIS-like pts, {wl.nx}x{wl.ny} grid, cell {wl.cell} m, "
                               f"h={wl.h} m, gaussian", "path": "oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} random cells x all {wl.n} points per step",
                         "extrapolated_full_grid_s": step_s * wl.nx * wl.ny / per_step},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
