"""Pins of the FP64 oracle helical cone-beam SF-TR projector and of the 26-neighbour regularizer.

Each pin checks the oracle against something other than itself:
* adjointness <A x, y> = <x, A' y> to 1e-12 (and the dense matrix, sampled
  rays and sampled voxels agree with forward/back);
* one slice, one detector row, no table feed and a voxel taller than the
  row's back-projection: the helical matrix equals the (separately pinned)
  2-D fan-beam matrix;
* a volume constant along z that covers every ray: each detector row sees
  the 2-D projection of the slice times 1/cos(cone angle of the row);
* A 1 against the exact length of each ray inside the volume box (slab
  intersection written here);
* A applied to rasterized ellipsoids converges, as voxels shrink, to their
  closed-form cell-averaged chord lengths on a two-turn helix (a wrong
  table feed or detector distance does not);
* the relaxed OS-LALM oracle on a small helical problem reaches the KKT
  point of the PWLS cost;
* the 26-neighbour regularizer against a brute-force sum over neighbour pairs.
"""

import math

import numpy as np
import pytest

import synth
from oracle import regularizer as reg
from oracle import solver as osolver
from oracle.helical import HelicalProjector
from oracle.projector import FanProjector


def _small(**kw):
    base = dict(nx=12, ny=10, nz=6, dx=2.0, dy=2.2, dz=1.5, ns=28, ds=2.0, nt=4, dt=2.4, na=30, dso=200.0,
                dsd=350.0, pitch=0.8, orbit_deg=720.0, orbit_start_deg=7.0, offset_x=0.3, offset_y=-0.2,
                offset_z=0.1, offset_s=0.25, offset_t=-0.15)
    base.update(kw)
    return synth.HelicalConeGeometry(**base)


def test_adjointness_fp64():
    g = _small()
    P = HelicalProjector(g)
    rng = np.random.default_rng(0)
    x = rng.random(P.shape)
    y = rng.random((g.na, g.nt, g.ns))
    lhs = float(np.sum(P.forward(x) * y))
    rhs = float(np.sum(x * P.back(y)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_matrix_rays_voxels_agree():
    g = _small(na=9)
    P = HelicalProjector(g)
    rng = np.random.default_rng(1)
    x = rng.random(P.shape)
    y = rng.random((g.na, g.nt, g.ns))
    views = np.array([4, 0, 7])
    A = P.matrix(views)
    np.testing.assert_allclose(A @ x.reshape(-1), P.forward(x, views).reshape(-1), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(A.T @ y[views].reshape(-1), P.back(y[views], views).reshape(-1), rtol=1e-12,
                               atol=1e-13)
    rv, rt, rs = rng.integers(0, g.na, 40), rng.integers(0, g.nt, 40), rng.integers(0, g.ns, 40)
    full = P.forward(x)
    np.testing.assert_allclose(P.forward_rays(x, rv, rt, rs), full[rv, rt, rs], rtol=1e-12, atol=1e-14)
    vox = rng.integers(0, P.nvox, 30)
    np.testing.assert_allclose(P.back_voxels(y, np.arange(g.na), vox), P.back(y).reshape(-1)[vox], rtol=1e-12,
                               atol=1e-14)


def test_single_row_reduces_to_fan_beam():
    """nz = nt = 1, pitch 0, voxel taller than the row's back-projection: R = 1, c = 1, A = A_2D."""
    g = _small(nz=1, nt=1, dz=20.0, pitch=0.0, offset_z=0.0, offset_t=0.0)
    P3 = HelicalProjector(g)
    P2 = FanProjector(g.transaxial())
    A3 = P3.matrix(np.arange(0, g.na, 3))
    A2 = P2.matrix(np.arange(0, g.na, 3))
    assert A3.shape == A2.shape
    np.testing.assert_allclose(A3, A2, rtol=1e-13, atol=1e-14)


def test_z_constant_volume_gives_cone_factor_times_fan_projection():
    g = _small(nz=60, dz=1.0, offset_z=0.0, pitch=0.5)
    # every column of every view must cover all rows: check the geometry before relying on it
    half_z = 0.5 * g.nz * g.dz
    zsrc = np.array([g.source_z(b) for b in g.betas()])
    mag_min = g.dsd / (g.dso + math.hypot(g.nx * g.dx, g.ny * g.dy) / 2)
    assert (half_z - np.abs(zsrc).max()) * mag_min > 0.5 * g.nt * g.dt + abs(g.offset_t) * g.dt + 1.0
    P3 = HelicalProjector(g)
    P2 = FanProjector(g.transaxial())
    x2 = np.random.default_rng(2).random((g.ny, g.nx))
    y3 = P3.forward(np.broadcast_to(x2, P3.shape))
    y2 = P2.forward(x2)
    ct = np.sqrt(1.0 + (g.row_heights() / g.dsd) ** 2)
    np.testing.assert_allclose(y3, ct[None, :, None] * y2[:, None, :], rtol=1e-12, atol=1e-14)


def _box_chord(g, sx, sy, sz, d):
    """Length of the line S + t d (d unit, t >= 0) inside the volume box."""
    lo = [(-g.nx / 2 + g.offset_x) * g.dx, (-g.ny / 2 + g.offset_y) * g.dy, (-g.nz / 2 + g.offset_z) * g.dz]
    hi = [lo[0] + g.nx * g.dx, lo[1] + g.ny * g.dy, lo[2] + g.nz * g.dz]
    t0, t1 = 0.0, np.inf
    for s, dd, a, b in zip((sx, sy, sz), d, lo, hi):
        if abs(dd) < 1e-15:
            if s < a or s > b:
                return 0.0
            continue
        ta, tb = (a - s) / dd, (b - s) / dd
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    return max(t1 - t0, 0.0)


def test_A1_matches_box_path_length():
    g = _small(nx=24, ny=24, nz=10, dx=1.0, dy=1.0, dz=1.0, ns=48, ds=1.4, nt=6, dt=1.5, na=16, offset_x=0.0,
               offset_y=0.0, offset_z=0.0, offset_s=0.0, offset_t=0.0)
    P = HelicalProjector(g)
    a1 = P.forward(np.ones(P.shape))
    n = 4
    q = (np.arange(n) + 0.5) / n - 0.5
    ref = np.zeros_like(a1)
    for v, b in enumerate(g.betas()):
        S = (-g.dso * math.cos(b), -g.dso * math.sin(b), g.source_z(b))
        for t, h in enumerate(g.row_heights()):
            for s, gm in enumerate(g.gammas()):
                acc = 0.0
                for qa in q:
                    for qb in q:
                        phi = b + gm + qa * g.dgamma
                        d = np.array([g.dsd * math.cos(phi), g.dsd * math.sin(phi), h + qb * g.dt])
                        acc += _box_chord(g, *S, d / np.linalg.norm(d))
                ref[v, t, s] = acc / n ** 2
    # rays that stay in the box for several voxels, away from its top and bottom faces
    inside = ref > 6.0
    rel = np.abs(a1[inside] - ref[inside]) / ref[inside]
    assert inside.sum() > 200
    assert np.median(rel) < 3e-3
    assert np.max(np.abs(a1 - ref)) < 1.5 * g.dx


def test_rasterized_phantom_converges_to_closed_form_chords():
    """A (rasterized ellipsoids) approaches their exact cell-averaged line integrals as voxels shrink,
    on a two-turn helix; a wrong table feed or detector distance stays far off."""
    S = [synth.Ellipsoid(3.0, -2.0, 1.0, 14.0, 10.0, 5.0, 0.3, 0.015),
         synth.Ellipsoid(-12.0, 8.0, -4.0, 7.0, 6.0, 3.0, 1.1, 0.01),
         synth.Ellipsoid(10.0, 10.0, 4.0, 6.0, 8.0, 3.5, 2.0, 0.012)]
    errs = []
    for f in (1, 2):
        g = synth.HelicalConeGeometry(nx=24 * f, ny=24 * f, nz=16 * f, dx=2.0 / f, dy=2.0 / f, dz=1.25 / f, ns=64,
                                      ds=2.0, nt=8, dt=2.2, na=40, dso=541.0, dsd=949.0, pitch=1.0, orbit_deg=720.0,
                                      orbit_start_deg=10.0)
        vol = synth.rasterize_solids(S, g, oversample=4, oversample_z=4)
        ya = synth.helical_line_integrals(S, g, n_sub=6)
        rel = lambda y: np.linalg.norm(y - ya) / np.linalg.norm(ya)  # noqa: E731
        errs.append(rel(HelicalProjector(g).forward(vol)))
    assert errs[1] < 0.4 * errs[0] and errs[1] < 0.025, errs
    assert rel(HelicalProjector(g.with_(pitch=1.2)).forward(vol)) > 5 * errs[1]
    assert rel(HelicalProjector(g.with_(dsd=1.05 * g.dsd)).forward(vol)) > 5 * errs[1]


def test_regularizer_directions_cover_26_neighbours():
    d = reg.DIRECTIONS_3D
    assert len(d) == 13
    both = set(d) | {tuple(-c for c in v) for v in d}
    assert len(both) == 26 and (0, 0, 0) not in both


@pytest.mark.parametrize("kind", ["hyperbola", "fair", "quadratic"])
def test_regularizer_3d_matches_brute_force_pairs(kind):
    rng = np.random.default_rng(5)
    nz, ny, nx = 3, 4, 5
    x = rng.random((nz, ny, nx)) * 0.1
    beta, delta = 1.7, 0.02
    phi, dphi, omega = reg.potential(kind, delta)
    val, grad, curv = 0.0, np.zeros_like(x), np.zeros_like(x)
    cells = [(k, j, i) for k in range(nz) for j in range(ny) for i in range(nx)]
    for p in cells:
        for q in cells:
            off = (q[2] - p[2], q[1] - p[1], q[0] - p[0])  # (dx, dy, dz)
            if max(abs(c) for c in off) != 1 or q <= p:  # each unordered neighbour pair once
                continue
            bi = beta / math.sqrt(sum(c * c for c in off))
            t = x[p] - x[q]
            val += bi * phi(t)
            grad[p] += bi * dphi(t)
            grad[q] -= bi * dphi(t)
            curv[p] += 2 * bi * omega(t)
            curv[q] += 2 * bi * omega(t)
    assert abs(reg.value(x, beta, delta, kind) - val) <= 1e-12 * abs(val)
    np.testing.assert_allclose(reg.gradient(x, beta, delta, kind), grad, rtol=1e-11, atol=1e-15)
    np.testing.assert_allclose(reg.curvature(x, beta, delta, kind), curv, rtol=1e-12)


def test_helical_solver_reaches_kkt_point():
    g = _small(nx=10, ny=10, nz=5, na=40, offset_x=0.0, offset_y=0.0, offset_z=0.0, offset_s=0.0, offset_t=0.0)
    P = HelicalProjector(g)
    S = [synth.Ellipsoid(0.0, 0.0, 0.0, 7.0, 6.0, 3.0, 0.2, 0.02)]
    y, w = synth.transmission_data(synth.helical_line_integrals(S, g, n_sub=2), 1e5, 5.0, 0)
    prob = osolver.PWLSProblem(P, y, w, beta=50.0, delta=1e-3)
    x = osolver.relaxed_os_lalm(prob, np.zeros(P.shape), M=4, alpha=1.999, n_iter=60)
    for _ in range(2):  # restarts: rho continuation starts again at 1
        x = osolver.relaxed_os_lalm(prob, x, M=1, alpha=1.999, n_iter=300)
    r = osolver.kkt_residual(prob, x)
    assert np.max(np.abs(r)) < 1e-6 * max(np.max(np.abs(x)), 1e-3)
