"""GPU FBP (ct_fbp) against the oracle FBP, and the solver's init_fbp option.

Tolerance: 1e-4 of the image maximum -- the FP32 filter sums a few hundred
terms of an alternating kernel and the back-projection interpolates at FP32
fan angles (~3e-5 cells), both well below the 1e-4 bound.
"""

import numpy as np
import pytest
import torch

import synth
from oracle.fbp import fbp_fan_arc

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("window", ["ramp", "hann"])
@pytest.mark.parametrize("gname", ["fan2d_128", "fan2d_512"])
def test_fbp_parity(window, gname):
    from paper_1512_04564_gb300 import ct

    c = synth.config_by_name(gname)
    g = c.geom
    d = synth.make_scan(c)
    y32 = d.y.astype(np.float32)
    G = ct.Geometry.from_fan(g)
    x = torch.empty(g.ny, g.nx, device="cuda")
    ct.ct_fbp(G, torch.from_numpy(y32).cuda(), x, window)
    torch.cuda.synchronize()
    ref = fbp_fan_arc(g, y32.astype(np.float64), window)
    assert np.max(np.abs(x.cpu().numpy() - ref)) <= 1e-4 * np.abs(ref).max()


def test_solver_init_fbp_equals_explicit_start():
    from paper_1512_04564_gb300 import ct

    c = synth.fan2d_128()
    g = c.geom
    d = synth.make_scan(c)
    G = ct.Geometry.from_fan(g)
    y = torch.from_numpy(d.y.astype(np.float32)).cuda()
    w = torch.from_numpy(d.w.astype(np.float32)).cuda()
    kw = dict(M=10, n_iter=3, alpha=1.999, beta=c.beta_per_mm, delta=c.delta)
    x1 = torch.zeros(g.ny, g.nx, device="cuda")
    ct.ct_relaxed_oslalm_solve(G, y, w, x1, init_fbp=True, **kw)
    x2 = torch.empty(g.ny, g.nx, device="cuda")
    ct.ct_fbp(G, y, x2, "hann")
    ct.ct_relaxed_oslalm_solve(G, y, w, x2, **kw)
    torch.cuda.synchronize()
    assert torch.equal(x1, x2)


def test_fbp_rejects_short_scan():
    from paper_1512_04564_gb300 import ct

    g = synth.FanArcGeometry(nx=32, ny=32, dx=1.0, dy=1.0, ns=64, ds=1.0, na=40, dso=300.0, dsd=500.0, orbit_deg=200.0)
    G = ct.Geometry.from_fan(g)
    with pytest.raises(ct.CTError) as e:
        ct.ct_fbp(G, torch.zeros(g.na, g.ns, device="cuda"), torch.empty(g.ny, g.nx, device="cuda"))
    assert e.value.status == ct.CT_ENOTSUP


@pytest.mark.parametrize("window", ["ramp", "hann"])
def test_helical_start_image_parity(window):
    """Helical scans: single-slice rebinning + fan-beam FBP per slice (ct_fbp on a helical geometry)
    against the oracle's fbp_helical_ssrb, within 1e-4 of the volume's maximum."""
    from oracle.fbp import fbp_helical_ssrb
    from paper_1512_04564_gb300 import ct

    c = synth.helix3d_64()
    g = c.geom
    d = synth.make_scan(c)
    y32 = d.y.astype(np.float32)
    G = ct.Geometry.from_helix(g)
    x = torch.empty(g.nz, g.ny, g.nx, device="cuda")
    ct.ct_fbp(G, torch.from_numpy(y32).cuda(), x, window)
    torch.cuda.synchronize()
    ref = fbp_helical_ssrb(g, y32.astype(np.float64), window)
    err = np.max(np.abs(x.cpu().numpy() - ref)) / np.abs(ref).max()
    print(f"helical FBP ({window}): max error {err:.2e} of the maximum")
    assert err <= 1e-4


def test_helical_solver_init_fbp_equals_explicit_start():
    from paper_1512_04564_gb300 import ct

    c = synth.helix3d_64()
    g = c.geom
    d = synth.make_scan(c)
    G = ct.Geometry.from_helix(g)
    y = torch.from_numpy(d.y.astype(np.float32)).cuda()
    w = torch.from_numpy(d.w.astype(np.float32)).cuda()
    kw = dict(M=8, n_iter=2, alpha=1.999, beta=c.beta_per_mm, delta=c.delta)
    x1 = torch.zeros(g.nz, g.ny, g.nx, device="cuda")
    ct.ct_relaxed_oslalm_solve(G, y, w, x1, init_fbp=True, **kw)
    x2 = torch.empty(g.nz, g.ny, g.nx, device="cuda")
    ct.ct_fbp(G, y, x2, "hann")
    ct.ct_relaxed_oslalm_solve(G, y, w, x2, **kw)
    torch.cuda.synchronize()
    assert torch.equal(x1, x2)
