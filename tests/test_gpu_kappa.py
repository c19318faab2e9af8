"""GPU parity of the regularizer's voxel weights kappa_n (Eq. (def_reg)).

* ct_kappa (kappa_j = sqrt([A'w]_j / [A'1]_j)) against the oracle's
  resolution_kappa: fan-beam with footprints on the fly and from the resident
  matrix (a short scan, so some pixels are met by no ray and get 0), and
  helical cone-beam.  kappa^2 is a ratio of two back-projections, each within
  the back-projector's rule (1e-5 of max(|value|, 1e-3 max)); at a pixel that
  a ray grazes, both are tiny and their ratio carries their relative errors,
  so the check weights kappa^2 by the pixel's coverage A'1: kappa^2 A'1
  (= A'w) within 3e-5 of the same rule, and kappa itself within 1e-5 where
  A'1 is at least 1% of its maximum;
* ct_reg_gradient with kappa, 8 neighbours (2-D) and 26 (3-D), against the
  oracle regularizer with kappa (1e-5 of the largest gradient; D_R 1e-5 per
  pixel);
* relaxed OS-LALM with kappa against the oracle after a fixed iteration count
  (RMSD <= 0.1 HU): 2-D, helical, and one slice of a batched launch.
"""

import numpy as np
import pytest
import torch

import synth
from oracle import regularizer as oreg
from oracle import solver as osolver
from oracle.helical import HelicalProjector
from oracle.projector import FanProjector

pytestmark = pytest.mark.gpu

MU_W = 0.02
HU = 1000.0 / MU_W
TOL = 1e-5


@pytest.fixture(scope="module")
def ct():
    from paper_1512_04564_gb300 import ct as ctmod

    return ctmod


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    return float(np.max(np.abs(got - ref) / den))


def _check_kappa(got, ref, den):
    got = got.astype(np.float64)
    assert rel_err(got ** 2 * den, ref ** 2 * den) <= 3 * TOL
    covered = den >= 1e-2 * den.max()
    assert covered.sum() > 0.5 * den.size
    assert np.max(np.abs(got[covered] - ref[covered]) / ref[covered]) <= TOL


SHORT = synth.FanArcGeometry(nx=45, ny=39, dx=1.0, dy=1.1, ns=40, ds=1.0, na=50, dso=90.0, dsd=150.0,
                             offset_x=0.3, offset_s=0.25, orbit_deg=60.0, orbit_start_deg=11.0)


def _weights(g, seed=0):
    E = [synth.Ellipse(0.0, 0.0, 0.35 * g.nx * g.dx, 0.3 * g.ny * g.dy, 0.2, 0.05),
         synth.Ellipse(2.0, -1.0, 3.0, 2.0, 0.0, 0.03)]
    _, w = synth.transmission_data(synth.fan_arc_line_integrals(E, g), 1e5, 5.0, seed)
    return w.astype(np.float32)


@pytest.mark.parametrize("resident", [False, True])
def test_kappa_fan_parity(ct, resident):
    g = SHORT
    w = _weights(g)
    G = ct.Geometry.from_fan(g)
    if resident:
        assert ct.ct_geom_precompute(G) > 0
    k = torch.empty(g.ny, g.nx, device="cuda")
    ct.ct_kappa(G, dev(w), k)
    torch.cuda.synchronize()
    P = FanProjector(g)
    ref = osolver.resolution_kappa(P, w.astype(np.float64))
    got = k.cpu().numpy()
    assert np.all(got[ref == 0] == 0) and (ref == 0).sum() > 0
    _check_kappa(got, ref, P.back(np.ones((g.na, g.ns))))


def test_kappa_helical_parity(ct):
    g = synth.HelicalConeGeometry(nx=40, ny=36, nz=20, dx=2.0, dy=2.2, dz=1.0, ns=72, ds=2.0, nt=8, dt=2.4, na=60,
                                  dso=300.0, dsd=520.0, pitch=0.8, orbit_deg=720.0, orbit_start_deg=7.0,
                                  offset_x=0.3, offset_y=-0.2, offset_z=0.1, offset_s=0.25, offset_t=-0.15)
    rng = np.random.default_rng(3)
    w = rng.uniform(2e4, 1e5, size=(g.na, g.nt, g.ns)).astype(np.float32)
    G = ct.Geometry.from_helix(g)
    k = torch.empty(g.nz, g.ny, g.nx, device="cuda")
    ct.ct_kappa(G, dev(w), k)
    torch.cuda.synchronize()
    P = HelicalProjector(g)
    ref = osolver.resolution_kappa(P, w.astype(np.float64))
    got = k.cpu().numpy()
    assert np.all(got[ref == 0] == 0)
    _check_kappa(got, ref, P.back(np.ones((g.na, g.nt, g.ns))))


@pytest.mark.parametrize("pot", ["hyperbola", "fair", "quadratic"])
def test_reg_gradient_kappa_2d(ct, pot):
    g = SHORT
    G = ct.Geometry.from_fan(g)
    rng = np.random.default_rng(8)
    x = (rng.random((g.ny, g.nx)) * 0.02).astype(np.float32)
    kappa = (200.0 + 100.0 * rng.random((g.ny, g.nx))).astype(np.float32)
    kappa[5, 7] = 0.0
    beta, delta = 3.0, 2e-4
    gr = torch.empty(g.ny, g.nx, device="cuda")
    cv = torch.empty_like(gr)
    ct.ct_reg_gradient(G, dev(x), beta, delta, pot, gr, cv, kappa=dev(kappa))
    torch.cuda.synchronize()
    x64, k64 = x.astype(np.float64), kappa.astype(np.float64)
    rg = oreg.gradient(x64, beta, delta, pot, k64)
    rc = oreg.curvature(x64, beta, delta, pot, k64)
    assert np.max(np.abs(gr.cpu().numpy() - rg)) <= TOL * np.abs(rg).max()
    assert rel_err(cv.cpu().numpy(), rc) <= TOL
    assert gr.cpu().numpy()[5, 7] == 0.0 and cv.cpu().numpy()[5, 7] == 0.0


@pytest.mark.parametrize("pot", ["hyperbola", "quadratic"])
def test_reg_gradient_kappa_3d(ct, pot):
    g = synth.HelicalConeGeometry(nx=37, ny=29, nz=11, dx=2.0, dy=2.2, dz=1.0, ns=72, ds=2.0, nt=8, dt=2.4, na=60,
                                  dso=300.0, dsd=520.0, pitch=0.8, orbit_deg=720.0)
    G = ct.Geometry.from_helix(g)
    rng = np.random.default_rng(9)
    x = (rng.random((g.nz, g.ny, g.nx)) * 0.02).astype(np.float32)
    kappa = (0.5 + rng.random((g.nz, g.ny, g.nx))).astype(np.float32)
    beta, delta = 3.0, 2e-4
    gr = torch.empty(g.nz, g.ny, g.nx, device="cuda")
    cv = torch.empty_like(gr)
    ct.ct_reg_gradient(G, dev(x), beta, delta, pot, gr, cv, kappa=dev(kappa))
    torch.cuda.synchronize()
    x64, k64 = x.astype(np.float64), kappa.astype(np.float64)
    rg = oreg.gradient(x64, beta, delta, pot, k64)
    rc = oreg.curvature(x64, beta, delta, pot, k64)
    assert np.max(np.abs(gr.cpu().numpy() - rg)) <= TOL * np.abs(rg).max()
    assert rel_err(cv.cpu().numpy(), rc) <= TOL


def _kappa_beta(beta, kappa):
    """beta divided by the mean kappa^2 over the pixels some ray meets, so the weighted penalty has the
    unweighted one's overall strength."""
    k2 = kappa[kappa > 0].astype(np.float64) ** 2
    return float(beta / k2.mean())


@pytest.mark.parametrize("resident", [False, True])
def test_solve_kappa_parity_fan2d_128(ct, resident):
    c = synth.fan2d_128()
    g = c.geom
    d = synth.make_scan(c)
    y32, w32 = d.y.astype(np.float32), d.w.astype(np.float32)
    P = FanProjector(g)
    k64 = osolver.resolution_kappa(P, w32.astype(np.float64))
    k32 = k64.astype(np.float32)
    beta = _kappa_beta(c.beta_per_mm, k64)
    M, n_iter = 10, 20
    prob = osolver.PWLSProblem(P, y32.astype(np.float64), w32.astype(np.float64), beta, c.delta, c.potential,
                               k32.astype(np.float64))
    xo = osolver.relaxed_os_lalm(prob, np.zeros((g.ny, g.nx)), M, 1.999, n_iter)
    G = ct.Geometry.from_fan(g)
    if resident:
        assert ct.ct_geom_precompute(G) > 0
    xg = torch.zeros(g.ny, g.nx, device="cuda")
    ct.ct_relaxed_oslalm_solve(G, dev(y32), dev(w32), xg, M=M, n_iter=n_iter, alpha=1.999, beta=beta, delta=c.delta,
                               potential=c.potential, kappa=dev(k32))
    mask = osolver.fov_mask(g)
    assert osolver.rmsd_hu(xg.cpu().numpy().astype(np.float64), xo, mask, c.hu_per_unit) <= 0.1
    # the weights change the result: the unweighted solve at the same overall strength differs
    xu = torch.zeros_like(xg)
    ct.ct_relaxed_oslalm_solve(G, dev(y32), dev(w32), xu, M=M, n_iter=n_iter, alpha=1.999, beta=beta * float(
        np.mean(k64[k64 > 0] ** 2)), delta=c.delta, potential=c.potential)
    assert osolver.rmsd_hu(xu.cpu().numpy().astype(np.float64), xo, mask, c.hu_per_unit) > 0.5


def test_solve_kappa_parity_helical(ct):
    g = synth.helix3d_64().geom
    S = synth.phantom_of(synth.helix3d_64(0))
    y, w = synth.transmission_data(synth.helical_line_integrals(S, g, n_sub=2), 1e5, 5.0, 0)
    y, w = y.astype(np.float32), w.astype(np.float32)
    P = HelicalProjector(g)
    k64 = osolver.resolution_kappa(P, w.astype(np.float64))
    k32 = k64.astype(np.float32)
    beta = _kappa_beta(2.0 ** 14 / MU_W ** 2, k64)
    delta = 10 * MU_W / 1000
    M, n_iter = 8, 3
    G = ct.Geometry.from_helix(g)
    kg = torch.empty(g.nz, g.ny, g.nx, device="cuda")
    ct.ct_kappa(G, dev(w), kg)
    x = torch.zeros(g.nz, g.ny, g.nx, device="cuda")
    ct.ct_relaxed_oslalm_solve(G, dev(y), dev(w), x, M=M, n_iter=n_iter, alpha=1.999, beta=beta, delta=delta,
                               kappa=kg)
    prob = osolver.PWLSProblem(P, y.astype(np.float64), w.astype(np.float64), beta, delta, "hyperbola",
                               k32.astype(np.float64))
    xo = osolver.relaxed_os_lalm(prob, np.zeros((g.nz, g.ny, g.nx)), M, 1.999, n_iter)
    d = osolver.rmsd_hu(x.cpu().numpy().astype(np.float64), xo, osolver.fov_mask(g), HU)
    assert d <= 0.1, d


def test_batched_kappa_slice_matches_oracle(ct):
    c = synth.fan2d_128()
    g = c.geom
    d = synth.make_scan(c)
    y32, w32 = d.y.astype(np.float32), d.w.astype(np.float32)
    P = FanProjector(g)
    k64 = osolver.resolution_kappa(P, w32.astype(np.float64))
    k32 = k64.astype(np.float32)
    beta = _kappa_beta(c.beta_per_mm, k64)
    G = ct.Geometry.from_fan(g)
    x1 = torch.zeros(g.ny, g.nx, device="cuda")
    x2 = torch.zeros(g.ny, g.nx, device="cuda")
    p = dict(M=10, n_iter=4, alpha=1.999, beta=beta, delta=c.delta)
    ct.ct_relaxed_oslalm_solve_batched([G, G], [dev(y32), dev(y32)], [dev(w32), dev(w32)], [x1, x2],
                                       [dict(kappa=dev(k32), **p), dict(**p)])
    prob = osolver.PWLSProblem(P, y32.astype(np.float64), w32.astype(np.float64), beta, c.delta, c.potential,
                               k32.astype(np.float64))
    xo = osolver.relaxed_os_lalm(prob, np.zeros((g.ny, g.nx)), 10, 1.999, 4)
    mask = osolver.fov_mask(g)
    assert osolver.rmsd_hu(x1.cpu().numpy().astype(np.float64), xo, mask, c.hu_per_unit) <= 0.1
    # the second slice (no kappa) is the unweighted problem
    assert osolver.rmsd_hu(x2.cpu().numpy().astype(np.float64), xo, mask, c.hu_per_unit) > 0.1
