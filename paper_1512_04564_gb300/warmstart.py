"""Learned warm start for relaxed OS-LALM.

Algorithm 1 starts from "an initial (FBP) image" (Sec. III-A).  This module
trains the tensor-core U-Net of include/ct_unet.h to map the FBP image of a
scan to the converged PWLS solution x* of the same scan, on pairs the solver
itself generates, and starts the solver from the network's output; the FBP
start remains the fallback.  Loss: image MSE (in units of water attenuation)
plus a data-consistency term 1/2 ||W^{1/2}(A x_hat - y)||^2 through the
differentiable projector (``autograd.project``).  All arithmetic runs in the
library's kernels (U-Net forward/backward/Adam, FBP, projectors, solver);
this module only sequences the calls.
"""

from __future__ import annotations

import math
import time

import torch

from . import autograd as _ag
from . import ct as _ct

MU_WATER = 0.02  # 1/mm


class UNetApply(torch.autograd.Function):
    """x_hat = U(x) with the library's forward; backward runs ct_unet_backward, which leaves the parameter
    gradients in the network (the anchor tensor only makes autograd call it)."""

    @staticmethod
    def forward(ctx, x, anchor, net):
        ctx.net = net
        return _ct.ct_unet_forward(net, x.contiguous())

    @staticmethod
    def backward(ctx, gy):
        _ct.ct_unet_backward(ctx.net, gy.contiguous().float())
        return None, torch.zeros(1, device=gy.device), None


def fbp_images(G, ys: torch.Tensor) -> torch.Tensor:
    """Hann-windowed FBP of each sinogram (the solver's plain initial image)."""
    out = torch.empty(ys.shape[0], G.ny, G.nx, device=ys.device)
    for i in range(ys.shape[0]):
        _ct.ct_fbp(G, ys[i], out[i], window="hann")
    return out


def solve_xstar(G, ys, ws, beta, delta, os_iters=20, m1_iters=40, M=20, alpha=1.999) -> torch.Tensor:
    """x* of each problem: relaxed OS-LALM from the FBP image (M subsets) followed by M = 1 iterations."""
    xs = torch.empty(ys.shape[0], G.ny, G.nx, device=ys.device)
    for i in range(ys.shape[0]):
        x = xs[i]
        _ct.ct_relaxed_oslalm_solve(G, ys[i], ws[i], x, M=M, n_iter=os_iters, alpha=alpha, beta=beta, delta=delta,
                                    init_fbp=True)
        if m1_iters:
            _ct.ct_relaxed_oslalm_solve(G, ys[i], ws[i], x, M=1, n_iter=m1_iters, alpha=alpha, beta=beta,
                                        delta=delta)
    return xs


def train(net, G, fbp, xstar, ys, ws, *, epochs=10, batch=8, lr=1e-3, lr_min=1e-4, lam_dc=1e-4, seed=0,
          log=None) -> list:
    """Adam on mean(((U(fbp) - x*)/mu_w)^2) + lam_dc * mean(w (A U(fbp) - y)^2) / mean(w); cosine learning rate.
    Returns the per-epoch mean losses."""
    n = fbp.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    anchor = torch.zeros(1, device=fbp.device, requires_grad=True)
    steps = epochs * math.ceil(n / batch)
    k = 0
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).tolist()
        tot = 0.0
        for s in range(0, n, batch):
            idx = perm[s:s + batch]
            xb, tb, yb, wb = fbp[idx], xstar[idx], ys[idx], ws[idx]
            xh = UNetApply.apply(xb, anchor, net)
            loss = ((xh - tb) / MU_WATER).pow(2).mean()
            if lam_dc > 0:
                r = _ag.project(xh, G) - yb
                loss = loss + lam_dc * (wb * r * r).mean() / wb.mean()
            loss.backward()
            cur = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * k / max(1, steps - 1)))
            _ct.ct_unet_adam(net, cur)
            tot += float(loss.detach()) * len(idx)
            k += 1
        hist.append(tot / n)
        if log:
            log(f"epoch {ep + 1}/{epochs}: loss {hist[-1]:.4g}")
    _ct.ct_unet_status(net)
    return hist


def warm_start(net, G, ys: torch.Tensor, batch: int = 8):
    """U-Net(FBP(y)) for each sinogram (inference) and the FBP images."""
    fbp = fbp_images(G, ys)
    out = torch.empty_like(fbp)
    for s in range(0, fbp.shape[0], batch):
        out[s:s + batch] = _ct.ct_unet_forward(net, fbp[s:s + batch].contiguous())
    return out, fbp


def evaluate(net, G, ys, ws, xstars, *, beta, delta, M=20, alpha=1.999, n_iter=40, tol_hu=1.0) -> dict:
    """Iterations and device seconds of relaxed OS-LALM to RMSD <= tol_hu vs x*, from the plain FBP start
    and from the warm start (which includes the FBP and the U-Net forward in its time)."""
    hu = 1000.0 / MU_WATER
    plain_it, plain_s, warm_it, warm_s, warm_rmsd0, fbp_rmsd0 = [], [], [], [], [], []
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    mask = None
    for i in range(ys.shape[0]):
        x = torch.zeros(G.ny, G.nx, device=ys.device)
        r = _ct.ct_relaxed_oslalm_solve(G, ys[i], ws[i], x, M=M, n_iter=n_iter, alpha=alpha, beta=beta, delta=delta,
                                        x_ref=xstars[i], hu_per_unit=hu, stop_rmsd_hu=tol_hu, init_fbp=True)
        plain_it.append(r["iters_done"] if r["seconds_to_tol"] > 0 else math.inf)
        plain_s.append(r["seconds_to_tol"] if r["seconds_to_tol"] > 0 else math.inf)
        e0.record(st)
        fb = torch.empty(1, G.ny, G.nx, device=ys.device)
        _ct.ct_fbp(G, ys[i], fb[0], window="hann")
        x0 = _ct.ct_unet_forward(net, fb)
        e1.record(st)
        torch.cuda.synchronize()
        t_ws = e0.elapsed_time(e1) * 1e-3
        if mask is None:  # the solver's RMSD region: the disk every view sees
            d = G.desc
            X = (torch.arange(G.nx, device=ys.device) - (G.nx - 1) / 2.0 + d.offset_x) * d.dx
            Y = (torch.arange(G.ny, device=ys.device) - (G.ny - 1) / 2.0 + d.offset_y) * d.dy
            half_fan = (d.ns / 2.0 + abs(d.offset_s)) * d.ds / d.dsd
            fov = min(d.dso * math.sin(min(half_fan, math.pi / 2)), min(G.nx * d.dx, G.ny * d.dy) / 2.0)
            mask = (X[None, :] ** 2 + Y[:, None] ** 2) <= fov ** 2
        warm_rmsd0.append(float(((x0[0] - xstars[i])[mask].double().pow(2).mean().sqrt()) * hu))
        fbp_rmsd0.append(float(((fb[0] - xstars[i])[mask].double().pow(2).mean().sqrt()) * hu))
        x = x0[0].contiguous()
        r = _ct.ct_relaxed_oslalm_solve(G, ys[i], ws[i], x, M=M, n_iter=n_iter, alpha=alpha, beta=beta, delta=delta,
                                        x_ref=xstars[i], hu_per_unit=hu, stop_rmsd_hu=tol_hu)
        warm_it.append(r["iters_done"] if r["seconds_to_tol"] > 0 else math.inf)
        warm_s.append(t_ws + r["seconds_to_tol"] if r["seconds_to_tol"] > 0 else math.inf)

    def stats(v):
        fin = [a for a in v if math.isfinite(a)]
        return {"mean": sum(fin) / len(fin) if fin else None, "median": sorted(fin)[len(fin) // 2] if fin else None,
                "reached": len(fin), "of": len(v)}

    return {"plain_iters": stats(plain_it), "warm_iters": stats(warm_it), "plain_seconds": stats(plain_s),
            "warm_seconds": stats(warm_s), "fbp_rmsd_hu": stats(fbp_rmsd0), "warm_start_rmsd_hu": stats(warm_rmsd0),
            "per_problem": {"plain_iters": plain_it, "warm_iters": warm_it}}


def timed(fn):
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0
