"""Pins of the FP64 oracle projector against facts that do not come from it.

The system matrix is the separable-footprint fan-beam A of the PWLS problem
(Sec. III, Eq. (ct_problem)).  Pins:
* adjointness <Ax, y> = <x, A'y> to 1e-12 (FP and BP must index one a_ij);
* parallel-beam limit: SF is exact there, so A equals the brute-force
  bin-averaged chord through each square pixel;
* fan beam: A within a few percent of the brute-force exact footprint;
* closed-form chords of uniform ellipses (error shrinks with the pixel size);
* A 1 against the analytic bin-averaged path length through the image box;
* sampled-ray / sampled-pixel / dense-matrix entry points agree with FP/BP.
"""

import math

import numpy as np
import pytest

import synth
from oracle.projector import FanProjector
from tests.exact_footprint import exact_box_path, exact_cell_weight

SMALL = synth.FanArcGeometry(nx=24, ny=20, dx=1.0, dy=1.0, ns=48, ds=1.2, na=30, dso=120.0, dsd=220.0,
                             offset_x=0.3, offset_y=-0.2, offset_s=0.25, orbit_start_deg=7.0)


def test_adjointness_fp64():
    P = FanProjector(SMALL)
    rng = np.random.default_rng(0)
    for trial in range(3):
        x = rng.standard_normal((SMALL.ny, SMALL.nx))
        y = rng.standard_normal((SMALL.na, SMALL.ns))
        a = float(np.sum(P.forward(x) * y))
        b = float(np.sum(x * P.back(y)))
        assert abs(a - b) <= 1e-12 * abs(a)


def test_views_subset_and_order():
    P = FanProjector(SMALL)
    rng = np.random.default_rng(1)
    x = rng.random((SMALL.ny, SMALL.nx))
    full = P.forward(x)
    views = np.array([17, 3, 29, 0])
    np.testing.assert_allclose(P.forward(x, views), full[views], rtol=0, atol=1e-13)
    y = rng.standard_normal((len(views), SMALL.ns))
    yfull = np.zeros((SMALL.na, SMALL.ns))
    yfull[views] = y
    np.testing.assert_allclose(P.back(y, views), P.back(yfull), rtol=0, atol=1e-12)


def test_matrix_rays_pixels_agree():
    P = FanProjector(SMALL)
    rng = np.random.default_rng(2)
    x = rng.random((SMALL.ny, SMALL.nx))
    views = np.array([2, 11, 19])
    A = P.matrix(views)
    np.testing.assert_allclose(A @ x.reshape(-1), P.forward(x, views).reshape(-1), rtol=1e-13, atol=1e-13)
    y = rng.standard_normal((len(views), SMALL.ns))
    np.testing.assert_allclose(A.T @ y.reshape(-1), P.back(y, views).reshape(-1), rtol=1e-13, atol=1e-12)
    rv = rng.integers(0, SMALL.na, 40)
    rb = rng.integers(0, SMALL.ns, 40)
    np.testing.assert_allclose(P.forward_rays(x, rv, rb), P.forward(x)[rv, rb], rtol=1e-13, atol=1e-13)
    pix = rng.integers(0, SMALL.nx * SMALL.ny, 30)
    np.testing.assert_allclose(P.back_pixels(y, views, pix), P.back(y, views).reshape(-1)[pix], rtol=1e-13, atol=1e-12)


def test_parallel_limit_equals_exact_footprint():
    """Far source: the footprint of a square pixel is an exact trapezoid of height l."""
    dso = 1.0e6
    g = synth.FanArcGeometry(nx=4, ny=4, dx=1.0, dy=1.0, ns=16, ds=0.8 * 2.0, na=3, dso=dso, dsd=2.0 * dso,
                             orbit_start_deg=11.0, orbit_deg=150.0)
    P = FanProjector(g)
    A = P.matrix()
    worst = 0.0
    for v in range(g.na):
        for s in range(g.ns):
            for iy in range(g.ny):
                for ix in range(g.nx):
                    ref = exact_cell_weight(g, v, s, ix, iy)
                    got = A[v * g.ns + s, iy * g.nx + ix]
                    worst = max(worst, abs(got - ref))
    assert worst < 1e-5, worst


def test_fan_footprint_close_to_exact():
    """Fan beam (4x4 image, 3 views): SF within 2% of the exact pixel shadow (max-normalised)."""
    g = synth.FanArcGeometry(nx=4, ny=4, dx=1.0, dy=1.0, ns=24, ds=0.6, na=3, dso=60.0, dsd=110.0,
                             orbit_start_deg=13.0, orbit_deg=240.0)
    P = FanProjector(g)
    A = P.matrix()
    E = np.zeros_like(A)
    for v in range(g.na):
        for s in range(g.ns):
            for iy in range(g.ny):
                for ix in range(g.nx):
                    E[v * g.ns + s, iy * g.nx + ix] = exact_cell_weight(g, v, s, ix, iy)
    assert np.max(np.abs(A - E)) < 0.02 * np.max(E)
    # both conserve the pixel's "mass": sum_s a_ij * dgamma ~ pixel area / distance
    rel = np.abs(A.sum(0) - E.sum(0)) / E.sum(0)
    assert np.max(rel) < 2e-3


def _ellipse_case(scale):
    g = synth.FanArcGeometry(nx=int(64 * scale), ny=int(64 * scale), dx=1.0 / scale, dy=1.0 / scale,
                             ns=96, ds=1.0, na=36, dso=300.0, dsd=500.0)
    E = [synth.Ellipse(2.0, -3.0, 18.0, 11.0, 0.4, 0.02), synth.Ellipse(-6.0, 5.0, 6.0, 4.0, -0.3, 0.01)]
    x = synth.rasterize_ellipses(E, g.nx, g.ny, g.dx, g.dy, oversample=8)
    return g, E, x


def test_closed_form_ellipse_chords_converge():
    errs = []
    for scale in (1, 2):
        g, E, x = _ellipse_case(scale)
        y = FanProjector(g).forward(x)
        ref = synth.fan_arc_line_integrals(E, g, n_gauss=16)
        errs.append(np.linalg.norm(y - ref) / np.linalg.norm(ref))
    # 1.3% at 1 mm pixels, 0.44% at 0.5 mm: pixelisation error, shrinking with the pixel size
    assert errs[0] < 0.02
    assert errs[1] < 0.5 * errs[0]


def test_disk_central_chord():
    """Uniform disk of radius R centred at the isocentre: the central ray's chord is 2R."""
    g = synth.FanArcGeometry(nx=128, ny=128, dx=0.5, dy=0.5, ns=65, ds=0.4, na=8, dso=400.0, dsd=700.0)
    R, mu = 20.0, 0.02
    x = synth.rasterize_ellipses([synth.Ellipse(0.0, 0.0, R, R, 0.0, mu)], g.nx, g.ny, g.dx, g.dy, oversample=16)
    y = FanProjector(g).forward(x)
    central = y[:, 32]  # gamma = 0 for ns odd and no offset
    # bin-averaged chord through the disk at fan angles within the central cell
    dg = g.dgamma
    gq, wq = np.polynomial.legendre.leggauss(16)
    d = 400.0 * np.sin(0.5 * dg * gq)
    ref = mu * 0.5 * np.sum(wq * 2.0 * np.sqrt(R * R - d * d))
    np.testing.assert_allclose(central, ref, rtol=3e-3)


def test_A1_matches_box_path_length():
    g = synth.FanArcGeometry(nx=32, ny=32, dx=1.0, dy=1.0, ns=64, ds=1.0, na=12, dso=150.0, dsd=260.0,
                             orbit_start_deg=3.0)
    P = FanProjector(g)
    a1 = P.forward(np.ones((g.ny, g.nx)))
    ref = np.array([[exact_box_path(g, v, s) for s in range(g.ns)] for v in range(g.na)])
    inside = ref > 0.5 * g.dx  # rays that cross more than a fraction of a pixel
    rel = np.abs(a1[inside] - ref[inside]) / ref[inside]
    assert np.median(rel) < 2e-3
    assert np.max(np.abs(a1 - ref)) < 0.5 * g.dx
    # half the pixel size, twice the pixels: the boundary error shrinks
    g2 = g.with_(nx=64, ny=64, dx=0.5, dy=0.5)
    a2 = FanProjector(g2).forward(np.ones((g2.ny, g2.nx)))
    assert np.max(np.abs(a2 - ref)) < 0.75 * np.max(np.abs(a1 - ref))


def test_amplitude_is_chord_through_centre():
    """A single centred pixel seen along a 45-degree ray: amplitude dx*sqrt(2) (pin of l)."""
    dso = 1.0e6
    g = synth.FanArcGeometry(nx=1, ny=1, dx=1.0, dy=1.0, ns=201, ds=0.02 * 2.0, na=1, dso=dso, dsd=2 * dso,
                             orbit_start_deg=45.0)
    P = FanProjector(g)
    a = P.forward(np.ones((1, 1)))[0]
    # at 45 degrees the footprint is a triangle of height sqrt(2) and half-width H = (sqrt(2)/2)/0.02 bins;
    # averaging it over the centred bin [-1/2, 1/2] gives sqrt(2) (1 - 1/(4H))
    H = (math.sqrt(2.0) / 2.0) / 0.02
    assert abs(a.max() - math.sqrt(2.0) * (1.0 - 0.25 / H)) < 1e-5
    # total "mass": sum_s a * (bin width at the pixel) = pixel area
    assert abs(a.sum() * 0.02 - 1.0) < 1e-6
