"""torch.autograd wrappers over the library's density, adjoint and LSCV kernels.

KDEGridFn: F = density(points, w, h) on the grid (Gaussian, split-FP16
tensor-core path with block-sparse skipping by default); backward runs
kde_grid_backward (dL/dpoints, dL/dw, dL/dh recomputed from the exponentials,
nothing stored).
LSCVFn: L = the grid least-squares cross-validation loss of F (kde_lscv_grid);
backward returns dL/dF and the loss's direct partials.
fit_bandwidth: Adam on (log h, weight logits) minimising the LSCV loss, the
quantitative counterpart of the paper's choice of bandwidth by eye (Sec. V-D),
with periodic checkpoints and resume.
"""
from __future__ import annotations

import math
import os

import torch

from . import FLAG_SKIP_ZERO, grid, grid_backward, lscv_grid


class KDEGridFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, points, weights, h, origin, cell, nx, ny, path="tc_split16"):
        hv = float(h)
        # on the tensor paths, skip the (tile, point) pairs whose products are
        # exactly zero in FP16: the same density, far fewer products at the
        # bandwidths a fit explores
        flags = FLAG_SKIP_ZERO if path in ("tc_split16", "tc_fp16") else 0
        F = grid(points.detach().contiguous(), weights.detach().contiguous(), origin, cell, nx, ny,
                 hv, "gaussian", path=path, flags=flags)
        ctx.save_for_backward(points, weights)
        ctx.hv, ctx.geom = hv, (origin, cell, nx, ny)
        ctx.h_like = h
        return F

    @staticmethod
    def backward(ctx, gF):
        points, weights = ctx.saved_tensors
        origin, cell, nx, ny = ctx.geom
        gxy, gw, gh = grid_backward(points.detach().contiguous(), weights.detach().contiguous(),
                                    origin, cell, nx, ny, ctx.hv, gF.contiguous())
        gh_t = torch.as_tensor(gh, dtype=ctx.h_like.dtype, device=ctx.h_like.device)
        return (gxy.to(points.dtype), gw.to(weights.dtype), gh_t, None, None, None, None, None)


class LSCVFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, F, points, weights, h, origin, cell, nx, ny):
        loss, G, gw, gxy, gh = lscv_grid(F.detach().contiguous(), points.detach().contiguous(),
                                         weights.detach().contiguous(), origin, cell, nx, ny,
                                         float(h))
        ctx.save_for_backward(G, gw, gxy)
        ctx.gh = gh
        ctx.h_like = h
        ctx.dtypes = (points.dtype, weights.dtype)
        return torch.as_tensor(loss, dtype=torch.float64, device=F.device)

    @staticmethod
    def backward(ctx, gL):
        G, gw, gxy = ctx.saved_tensors
        g = gL.to(torch.float32)
        gh_t = torch.as_tensor(ctx.gh, dtype=ctx.h_like.dtype, device=ctx.h_like.device) * gL.to(
            ctx.h_like.dtype)
        return (G * g, (gxy * g).to(ctx.dtypes[0]), (gw * g).to(ctx.dtypes[1]), gh_t,
                None, None, None, None)


def density(points, weights, h, origin, cell, nx, ny, path="tc_split16"):
    """Differentiable F[j, i] (Gaussian) with respect to points, weights and h."""
    return KDEGridFn.apply(points, weights, h, origin, cell, nx, ny, path)


def lscv_loss(points, weights, h, origin, cell, nx, ny, path="tc_split16"):
    """Differentiable grid LSCV loss of the Gaussian density."""
    F = density(points, weights, h, origin, cell, nx, ny, path)
    return LSCVFn.apply(F, points, weights, h, origin, cell, nx, ny)


def fit_bandwidth(points, weights0, origin, cell, nx, ny, h0, steps=200, lr=0.05,
                  checkpoint=None, every=20, resume=True, path="tc_split16", log=None):
    """Minimise the LSCV loss over theta = (log h, omega), w = N softmax(omega).

    points: [n,2] float64 cuda; weights0: [n] initial weights (e.g. how many
    raw fixes each kept fix stands for).  Saves (theta, Adam state, step) to
    `checkpoint` every `every` steps and resumes from it when present.
    Returns (h, weights, losses).
    """
    dev = points.device
    n = points.shape[0]
    log_h = torch.tensor(math.log(h0), dtype=torch.float64, device=dev, requires_grad=True)
    omega = torch.log(weights0.to(torch.float64).clamp_min(1e-30)).clone().detach()
    omega.requires_grad_(True)
    opt = torch.optim.Adam([log_h, omega], lr=lr)
    start, losses = 0, []
    if checkpoint and resume and os.path.exists(checkpoint):
        st = torch.load(checkpoint, map_location=dev)
        with torch.no_grad():
            log_h.copy_(st["log_h"])
            omega.copy_(st["omega"])
        opt.load_state_dict(st["opt"])
        start, losses = int(st["step"]), list(st["losses"])
    for step in range(start, steps):
        opt.zero_grad(set_to_none=True)
        # the logits stay FP64 for Adam; the softmax runs in FP32 (the weights
        # are FP32 for the kernels anyway)
        w = n * torch.softmax(omega.to(torch.float32), dim=0)
        L = lscv_loss(points, w, torch.exp(log_h), origin, cell, nx, ny, path)
        L.backward()
        opt.step()
        losses.append(float(L))
        if log:
            log(step, float(L), float(torch.exp(log_h)))
        if checkpoint and ((step + 1) % every == 0 or step + 1 == steps):
            tmp = checkpoint + ".tmp"
            torch.save({"log_h": log_h.detach(), "omega": omega.detach(),
                        "opt": opt.state_dict(), "step": step + 1, "losses": losses}, tmp)
            os.replace(tmp, checkpoint)
    w = n * torch.softmax(omega.detach().to(torch.float32), dim=0)
    return float(torch.exp(log_h.detach())), w, losses
