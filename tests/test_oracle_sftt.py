"""Pins of the oracle's trapezoid axial footprint (SF-TT) for helical cone-beam.

* adjointness <A x, y> = <x, A' y> to 1e-12;
* the axial factor equals the mean, over the magnifications dsd / L with L
  between the nearest and the farthest corner of the voxel's column, of the
  rectangle footprint's row overlap (an average of rectangles, integrated
  here by a fine midpoint rule; the transaxial factor l_xy c_t T(s) is taken
  from the rectangle model's matrix, pinned on its own);
* the row sum of the axial factor is the closed form
  (dz dsd / dt) (1/L_min + 1/L_max) / 2, i.e. L (1/L_min + 1/L_max) / 2 times
  the rectangle model's;
* a volume constant along z that covers every ray projects exactly as with
  the rectangle model (the voxels' trapezoids tile each column);
* A applied to rasterized ellipsoids converges, as voxels shrink, to their
  closed-form cell-averaged chord lengths.
"""

import math

import numpy as np

import synth
from oracle.helical import HelicalProjector


def _small(**kw):
    base = dict(nx=12, ny=10, nz=6, dx=2.0, dy=2.2, dz=1.5, ns=28, ds=2.0, nt=4, dt=2.4, na=30, dso=200.0,
                dsd=350.0, pitch=0.8, orbit_deg=720.0, orbit_start_deg=7.0, offset_x=0.3, offset_y=-0.2,
                offset_z=0.1, offset_s=0.25, offset_t=-0.15)
    base.update(kw)
    return synth.HelicalConeGeometry(**base)


def test_adjointness_fp64():
    g = _small(axial="trap")
    P = HelicalProjector(g)
    rng = np.random.default_rng(0)
    x = rng.random(P.shape)
    y = rng.random((g.na, g.nt, g.ns))
    lhs = float(np.sum(P.forward(x) * y))
    rhs = float(np.sum(x * P.back(y)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _column(g, beta, ix, iy):
    """Transaxial source distances of the column's centre and of its nearest and farthest corners."""
    xc = (ix - (g.nx - 1) / 2 + g.offset_x) * g.dx
    yc = (iy - (g.ny - 1) / 2 + g.offset_y) * g.dy
    sx, sy = -g.dso * math.cos(beta), -g.dso * math.sin(beta)
    L = math.hypot(xc - sx, yc - sy)
    corners = [math.hypot(xc + 0.5 * a * g.dx - sx, yc + 0.5 * b * g.dy - sy) for a in (-1, 1) for b in (-1, 1)]
    return L, min(corners), max(corners)


def _row_overlap(u0, u1, t):
    return max(0.0, min(u1, t + 0.5) - max(u0, t - 0.5))


def _axial(g, beta, iz, L, Lmin, Lmax, n=20000):
    """(R_rect(t), R_trap(t)) for every row t: the rectangle at magnification dsd/L, and the mean of
    rectangles over magnifications m uniform in [dsd/Lmax, dsd/Lmin]."""
    zc = (iz - (g.nz - 1) / 2 + g.offset_z) * g.dz
    z0, z1 = zc - 0.5 * g.dz - g.source_z(beta), zc + 0.5 * g.dz - g.source_z(beta)
    c = (g.nt - 1) / 2 - g.offset_t

    def rows(m):
        return z0 * m / g.dt + c, z1 * m / g.dt + c

    rr = np.array([_row_overlap(*rows(g.dsd / L), t) for t in range(g.nt)])
    m_lo, m_hi = g.dsd / Lmax, g.dsd / Lmin
    ms = m_lo + (np.arange(n) + 0.5) / n * (m_hi - m_lo)
    rt = np.zeros(g.nt)
    for m in ms:
        u0, u1 = rows(m)
        rt += [_row_overlap(u0, u1, t) for t in range(g.nt)]
    return rr, rt / n


def test_trapezoid_is_mean_of_rectangles():
    g = _small(dz=1.2, dt=1.3, nt=6, dso=60.0, dsd=110.0, nx=8, ny=8, ns=40, na=12, orbit_deg=360.0)
    gt = g.with_(axial="trap")
    views = np.arange(0, g.na, 3)
    A_r = HelicalProjector(g).matrix(views)
    A_t = HelicalProjector(gt).matrix(views)
    ct = np.sqrt(1.0 + (g.row_heights() / g.dsd) ** 2)
    betas = g.betas()
    checked = 0
    for k, v in enumerate(views):
        for (ix, iy, iz) in [(1, 2, 2), (4, 4, 3), (6, 1, 0), (3, 6, 5)]:
            j = (iz * g.ny + iy) * g.nx + ix
            L, Lmin, Lmax = _column(g, betas[v], ix, iy)
            rr, rt = _axial(g, betas[v], iz, L, Lmin, Lmax)
            if rr.max() <= 0:
                continue
            tref = int(np.argmax(rr))
            for s in range(g.ns):
                row = lambda t: (k * g.nt + t) * g.ns + s  # noqa: E731
                w = A_r[row(tref), j] / (ct[tref] * rr[tref])  # l_xy T_j(s) from the rectangle model
                for t in range(g.nt):
                    want = w * ct[t] * rt[t]
                    assert abs(A_t[row(t), j] - want) <= 1e-7 * max(w, 1e-12), (v, ix, iy, iz, t, s)
                    checked += w > 0
    assert checked > 100


def test_row_sum_closed_form():
    g = _small(nz=3, dz=0.8, nt=16, dt=1.0, offset_z=0.0, offset_t=0.0, pitch=0.1)
    gt = g.with_(axial="trap")
    views = np.arange(0, g.na, 5)
    A_r = HelicalProjector(g).matrix(views)
    A_t = HelicalProjector(gt).matrix(views)
    ct = np.sqrt(1.0 + (g.row_heights() / g.dsd) ** 2)
    betas = g.betas()
    n = 0
    for k, v in enumerate(views):
        for ix, iy in [(0, 0), (5, 4), (11, 9), (7, 2)]:
            j = (1 * g.ny + iy) * g.nx + ix
            L, Lmin, Lmax = _column(g, betas[v], ix, iy)
            blk = lambda A: A[k * g.nt * g.ns:(k + 1) * g.nt * g.ns, j].reshape(g.nt, g.ns)  # noqa: E731
            sr = (blk(A_r) / ct[:, None]).sum(axis=0)
            st = (blk(A_t) / ct[:, None]).sum(axis=0)
            # the voxel's shadow must lie inside the detector rows
            assert blk(A_t)[0].max() == 0 and blk(A_t)[-1].max() == 0
            m = sr > 1e-9 * sr.max()
            np.testing.assert_allclose(st[m] / sr[m], L * (1 / Lmin + 1 / Lmax) / 2, rtol=1e-12)
            n += m.sum()
    assert n > 20


def test_z_constant_volume_matches_rectangle_model():
    g = _small(nz=60, dz=1.0, offset_z=0.0, pitch=0.5)
    half_z = 0.5 * g.nz * g.dz
    zsrc = np.array([g.source_z(b) for b in g.betas()])
    mag_min = g.dsd / (g.dso + math.hypot(g.nx * g.dx, g.ny * g.dy) / 2)
    assert (half_z - np.abs(zsrc).max()) * mag_min > 0.5 * g.nt * g.dt + abs(g.offset_t) * g.dt + 1.0
    x2 = np.random.default_rng(2).random((g.ny, g.nx))
    vol = np.broadcast_to(x2, (g.nz, g.ny, g.nx))
    yr = HelicalProjector(g).forward(vol)
    yt = HelicalProjector(g.with_(axial="trap")).forward(vol)
    np.testing.assert_allclose(yt, yr, rtol=1e-12, atol=1e-14)
    # but not voxel by voxel: a z-varying volume projects differently
    xv = np.random.default_rng(3).random((g.nz, g.ny, g.nx))
    d = HelicalProjector(g.with_(axial="trap")).forward(xv) - HelicalProjector(g).forward(xv)
    assert np.abs(d).max() > 1e-6 * np.abs(yr).max()


def test_rasterized_phantom_converges_to_closed_form_chords():
    S = [synth.Ellipsoid(3.0, -2.0, 1.0, 14.0, 10.0, 5.0, 0.3, 0.015),
         synth.Ellipsoid(-12.0, 8.0, -4.0, 7.0, 6.0, 3.0, 1.1, 0.01),
         synth.Ellipsoid(10.0, 10.0, 4.0, 6.0, 8.0, 3.5, 2.0, 0.012)]
    errs = []
    for f in (1, 2):
        g = synth.HelicalConeGeometry(nx=24 * f, ny=24 * f, nz=16 * f, dx=2.0 / f, dy=2.0 / f, dz=1.25 / f, ns=64,
                                      ds=2.0, nt=8, dt=2.2, na=40, dso=541.0, dsd=949.0, pitch=1.0, orbit_deg=720.0,
                                      orbit_start_deg=10.0, axial="trap")
        vol = synth.rasterize_solids(S, g, oversample=4, oversample_z=4)
        ya = synth.helical_line_integrals(S, g, n_sub=6)
        errs.append(np.linalg.norm(HelicalProjector(g).forward(vol) - ya) / np.linalg.norm(ya))
    assert errs[1] < 0.4 * errs[0] and errs[1] < 0.025, errs
