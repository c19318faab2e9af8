"""The SF projector pair as a differentiable PyTorch operation.

``project(x, geom)`` computes y = A x with the library's forward projector;
its backward is the matched back-projector, grad_x = A' grad_y (the same
a_ij), so data-consistency terms such as 1/2 ||W^{1/2}(A x - y)||^2 can be
trained through (Sec. III, Eq. (ct_problem): A is the system matrix).
Both directions run in the CUDA library; this module only marshals tensors.
Images may carry a leading batch dimension: [B, ny, nx] -> [B, nviews, ns].
"""

from __future__ import annotations

import torch

from . import ct as _ct


class ForwardProjection(torch.autograd.Function):
    """y = A_V x; backward grad_x = A_V' grad_y (hand-written adjoint)."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, geom: "_ct.Geometry", views):
        nv = geom.na if views is None else len(views)
        xs = x.reshape(-1, geom.ny, geom.nx).contiguous()
        y = torch.empty(xs.shape[0], nv, geom.ns, device=x.device, dtype=torch.float32)
        for b in range(xs.shape[0]):
            _ct.ct_forward(geom, xs[b], y[b], views=views)
        ctx.geom, ctx.views, ctx.shape = geom, views, x.shape
        return y.reshape(*x.shape[:-2], nv, geom.ns)

    @staticmethod
    def backward(ctx, gy: torch.Tensor):
        geom, views = ctx.geom, ctx.views
        nv = geom.na if views is None else len(views)
        gys = gy.reshape(-1, nv, geom.ns).contiguous().float()
        gx = torch.empty(gys.shape[0], geom.ny, geom.nx, device=gy.device, dtype=torch.float32)
        for b in range(gys.shape[0]):
            _ct.ct_back(geom, gys[b], gx[b], views=views)
        return gx.reshape(ctx.shape), None, None


class BackProjection(torch.autograd.Function):
    """x = A_V' y; backward grad_y = A_V grad_x."""

    @staticmethod
    def forward(ctx, y: torch.Tensor, geom: "_ct.Geometry", views):
        nv = geom.na if views is None else len(views)
        ys = y.reshape(-1, nv, geom.ns).contiguous()
        x = torch.empty(ys.shape[0], geom.ny, geom.nx, device=y.device, dtype=torch.float32)
        for b in range(ys.shape[0]):
            _ct.ct_back(geom, ys[b], x[b], views=views)
        ctx.geom, ctx.views, ctx.shape = geom, views, y.shape
        return x.reshape(*y.shape[:-2], geom.ny, geom.nx)

    @staticmethod
    def backward(ctx, gx: torch.Tensor):
        geom, views = ctx.geom, ctx.views
        nv = geom.na if views is None else len(views)
        gxs = gx.reshape(-1, geom.ny, geom.nx).contiguous().float()
        gy = torch.empty(gxs.shape[0], nv, geom.ns, device=gx.device, dtype=torch.float32)
        for b in range(gxs.shape[0]):
            _ct.ct_forward(geom, gxs[b], gy[b], views=views)
        return gy.reshape(ctx.shape), None, None


def project(x: torch.Tensor, geom: "_ct.Geometry", views=None) -> torch.Tensor:
    """Differentiable forward projection A_V x."""
    return ForwardProjection.apply(x, geom, views)


def backproject(y: torch.Tensor, geom: "_ct.Geometry", views=None) -> torch.Tensor:
    """Differentiable back-projection A_V' y."""
    return BackProjection.apply(y, geom, views)
