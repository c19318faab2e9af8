"""Pins of the oracle's fan-beam FBP (the initial image of Algorithm 1).

* a uniform disk's analytic projections reconstruct to its value (both windows),
  off-centre too, and the exterior to zero;
* the FBP of a noiseless ellipse phantom is close to the rasterized phantom
  (edges blur by the interpolation and window: < 20 HU RMS in the FOV).
"""

import math

import numpy as np

import synth
from oracle.fbp import fbp_fan_arc


def test_disk_value_both_windows():
    g = synth.FanArcGeometry(nx=128, ny=128, dx=0.5, dy=0.5, ns=301, ds=0.6, na=360, dso=300.0, dsd=500.0)
    sino = synth.fan_arc_line_integrals([synth.Ellipse(0, 0, 20, 20, 0, 0.02)], g)
    X = (np.arange(128) - 63.5) * 0.5
    R = np.hypot(X[None, :], X[:, None])
    for win in ("ramp", "hann"):
        img = fbp_fan_arc(g, sino, win)
        assert abs(img[R < 15].mean() - 0.02) < 2e-5
        assert abs(img[R > 25].mean()) < 2e-5


def test_offcentre_disk():
    g = synth.FanArcGeometry(nx=128, ny=128, dx=0.5, dy=0.5, ns=301, ds=0.6, na=360, dso=300.0, dsd=500.0)
    sino = synth.fan_arc_line_integrals([synth.Ellipse(8.0, -5.0, 10, 10, 0, 0.01)], g)
    X = (np.arange(128) - 63.5) * 0.5
    R = np.hypot(X[None, :] - 8.0, X[:, None] + 5.0)
    img = fbp_fan_arc(g, sino, "ramp")
    assert abs(img[R < 6].mean() - 0.01) < 2e-5


def test_phantom_close_to_truth():
    c = synth.fan2d_128()
    li = synth.fan_arc_line_integrals(synth.random_ellipses_cfg1(0), c.geom)
    img = fbp_fan_arc(c.geom, li, "hann")
    truth = synth.rasterize_ellipses(synth.random_ellipses_cfg1(0), 128, 128, 1.0, 1.0)
    from oracle.solver import fov_mask

    m = fov_mask(c.geom)
    rms_hu = math.sqrt(float(np.mean((img - truth)[m] ** 2))) * 5e4
    assert rms_hu < 20.0


# ---- helical start image: single-slice rebinning + fan-beam FBP (the paper gives no helical FBP)

def _z(g, k):
    return (k - (g.nz - 1) / 2.0 + g.offset_z) * g.dz


def test_ssrb_z_constant_scan_is_the_fan_sinogram():
    """A volume constant in z projects every row to the transaxial line integral over the cosine of
    the row's cone angle; rebinning must return the 2-D fan sinogram of the slice's one-turn window,
    whose source heights are centred on the slice."""
    from oracle.fbp import ssrb_sinogram

    g = synth.helix3d_64().geom
    E = [synth.Ellipse(3.0, -4.0, 30.0, 22.0, 0.4, 0.02), synth.Ellipse(-10.0, 6.0, 8.0, 8.0, 0.0, 0.01)]
    p2 = synth.fan_arc_line_integrals(E, g.transaxial(), n_gauss=2)  # [na][ns] over both turns
    h = g.row_heights()
    sino = p2[:, None, :] * (np.hypot(g.dsd, h) / g.dsd)[None, :, None]
    na_turn = g.na // 2
    cover = g.nt * g.dt * g.dso / g.dsd
    zsrc = np.array([g.source_z(b) for b in g.betas()])
    for k in range(g.nz):
        v0, p = ssrb_sinogram(g, sino, k)
        assert p.shape == (na_turn, g.ns) and 0 <= v0 <= g.na - na_turn
        # exact up to the linear interpolation of the rows' cone-angle secant, 1 + h^2 / (2 dsd^2):
        # at most dt^2 / (8 dsd^2) relative
        np.testing.assert_allclose(p, p2[v0:v0 + na_turn], rtol=g.dt ** 2 / (4 * g.dsd ** 2),
                                   atol=1e-12 * np.abs(p2).max())
        if abs(_z(g, k)) <= 0.5 * g.pitch * cover * (g.orbit_deg / 360.0 - 1.0):  # window not clipped
            assert abs(zsrc[v0 + na_turn // 2] - _z(g, k)) <= abs(zsrc[1] - zsrc[0])


def test_ssrb_fbp_of_z_constant_scan_is_fan_fbp():
    from oracle.fbp import fbp_helical_ssrb, ssrb_sinogram

    g = synth.helix3d_64().geom
    E = [synth.Ellipse(0.0, 0.0, 35.0, 30.0, 0.2, 0.018)]
    p2 = synth.fan_arc_line_integrals(E, g.transaxial(), n_gauss=2)
    sino = p2[:, None, :] * (np.hypot(g.dsd, g.row_heights()) / g.dsd)[None, :, None]
    vol = fbp_helical_ssrb(g, sino, "hann")
    for k in (0, 7, 15):
        v0, _ = ssrb_sinogram(g, sino, k)
        g2 = g.transaxial().with_(na=g.na // 2, orbit_deg=360.0, orbit_start_deg=v0 * g.orbit_deg / g.na)
        ref = fbp_fan_arc(g2, p2[v0:v0 + g.na // 2], "hann")
        np.testing.assert_allclose(vol[k], ref, rtol=0, atol=g.dt ** 2 / (4 * g.dsd ** 2) * np.abs(ref).max())
    X = (np.arange(g.nx) - (g.nx - 1) / 2.0) * g.dx
    R = np.hypot(X[None, :], X[:, None])
    assert abs(vol[7][R < 20].mean() - 0.018) < 0.02 * 0.018


def test_ssrb_fbp_places_a_cylinder_in_its_slices():
    """An elliptic cylinder between z = 1 and 6.5 mm (analytic helical line integrals) shows up at
    its value in the fully covered slices inside it and not in the slices below it: a wrong row
    mapping or a flipped source height would move it."""
    from oracle.fbp import fbp_helical_ssrb

    g = synth.helix3d_64().geom
    cyl = synth.phantom3d.EllipticCylinder(cx=4.0, cy=-3.0, a=30.0, b=25.0, theta=0.3, z0=1.0, z1=6.5, value=0.02)
    sino = synth.helical_line_integrals([cyl], g, n_sub=2)
    vol = fbp_helical_ssrb(g, sino, "hann")
    X = (np.arange(g.nx) - (g.nx - 1) / 2.0) * g.dx
    inside = np.hypot((X[None, :] - 4.0) / 30.0, (X[:, None] + 3.0) / 25.0) < 0.6
    cover = g.nt * g.dt * g.dso / g.dsd
    full = lambda k: abs(_z(g, k)) <= 0.5 * g.pitch * cover * (g.orbit_deg / 360.0 - 1.0) + 1e-9  # noqa: E731
    ins = [k for k in range(g.nz) if 2.5 <= _z(g, k) <= 5.0 and full(k)]
    out = [k for k in range(g.nz) if _z(g, k) <= -1.0 and full(k)]
    assert ins and out
    for k in ins:
        assert abs(vol[k][inside].mean() - 0.02) < 0.05 * 0.02, (k, vol[k][inside].mean())
    for k in out:
        assert abs(vol[k][inside].mean()) < 0.05 * 0.02, (k, vol[k][inside].mean())
