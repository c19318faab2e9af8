"""The projector as a torch.autograd.Function: its backward is the hand-written adjoint.

Checks: the gradient of <A x, v> equals the FP64 oracle's A'v; the gradient of
the weighted data-consistency loss 1/2 ||W^{1/2}(A x - y)||^2 matches central
finite differences of the same loss evaluated by the FP64 oracle; batched
inputs match per-slice calls; back-projection's gradient is the forward
projection.
"""

import numpy as np
import pytest
import torch

import synth
from oracle.projector import FanProjector

pytestmark = pytest.mark.gpu

G_SMALL = synth.FanArcGeometry(nx=40, ny=36, dx=1.0, dy=1.0, ns=72, ds=1.0, na=30, dso=300.0, dsd=500.0,
                               offset_x=0.25, orbit_start_deg=5.0)


@pytest.fixture(scope="module")
def mods():
    from paper_1512_04564_gb300 import autograd as ag
    from paper_1512_04564_gb300 import ct

    return ct, ag


def _rel(got, ref):
    den = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    return float(np.max(np.abs(got - ref) / den))


@pytest.mark.parametrize("views", [None, [3, 11, 29, 0]])
def test_gradient_of_inner_product_is_oracle_adjoint(mods, views):
    ct, ag = mods
    g = G_SMALL
    G = ct.Geometry.from_fan(g)
    rng = np.random.default_rng(0)
    nv = g.na if views is None else len(views)
    x = torch.from_numpy(rng.random((g.ny, g.nx)).astype(np.float32)).cuda().requires_grad_(True)
    v = rng.random((nv, g.ns)).astype(np.float32)
    y = ag.project(x, G, views)
    (y * torch.from_numpy(v).cuda()).sum().backward()
    ref = FanProjector(g).back(v.astype(np.float64), views)
    assert _rel(x.grad.cpu().numpy(), ref) <= 1e-5


def test_data_consistency_gradient_vs_oracle_finite_differences(mods):
    ct, ag = mods
    g = G_SMALL
    G = ct.Geometry.from_fan(g)
    P = FanProjector(g)
    E = [synth.Ellipse(0.0, 0.0, 14.0, 11.0, 0.3, 0.02), synth.Ellipse(3.0, -2.0, 4.0, 3.0, 0.0, 0.005)]
    y, w = synth.transmission_data(synth.fan_arc_line_integrals(E, g), 1e5, 5.0, seed=3)
    y32, w32 = y.astype(np.float32), (w / 1e4).astype(np.float32)
    rng = np.random.default_rng(1)
    x0 = (synth.rasterize_ellipses(E, g.nx, g.ny, g.dx, g.dy, g.offset_x, g.offset_y, oversample=2)
          + 0.002 * rng.standard_normal((g.ny, g.nx))).astype(np.float32)
    x = torch.from_numpy(x0).cuda().requires_grad_(True)
    yd, wd = torch.from_numpy(y32).cuda(), torch.from_numpy(w32).cuda()
    loss = 0.5 * (wd * (ag.project(x, G) - yd) ** 2).sum()
    loss.backward()
    grad = x.grad.cpu().numpy().astype(np.float64)

    def f64(xx):
        r = P.forward(xx) - y32.astype(np.float64)
        return 0.5 * float(np.sum(w32.astype(np.float64) * r * r))

    x64 = x0.astype(np.float64)
    for trial in range(4):
        d = rng.standard_normal((g.ny, g.nx))
        eps = 1e-4
        fd = (f64(x64 + eps * d) - f64(x64 - eps * d)) / (2 * eps)
        assert abs(float(np.sum(grad * d)) - fd) <= 1e-4 * max(abs(fd), 1e-3 * np.linalg.norm(grad) * np.linalg.norm(d))


def test_batched_matches_per_slice(mods):
    ct, ag = mods
    g = G_SMALL
    G = ct.Geometry.from_fan(g)
    xb = torch.rand(3, g.ny, g.nx, device="cuda")
    yb = ag.project(xb, G)
    for b in range(3):
        ys = torch.empty(g.na, g.ns, device="cuda")
        ct.ct_forward(G, xb[b].contiguous(), ys)
        assert torch.equal(yb[b], ys)
    assert yb.shape == (3, g.na, g.ns)


def test_backprojection_gradient_is_projection(mods):
    ct, ag = mods
    g = G_SMALL
    G = ct.Geometry.from_fan(g)
    yv = torch.rand(g.na, g.ns, device="cuda", requires_grad=True)
    u = torch.rand(g.ny, g.nx, device="cuda")
    (ag.backproject(yv, G) * u).sum().backward()
    Au = torch.empty(g.na, g.ns, device="cuda")
    ct.ct_forward(G, u, Au)
    assert torch.allclose(yv.grad, Au, rtol=0, atol=0)
