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
