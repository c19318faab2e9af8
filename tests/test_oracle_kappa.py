"""Pins of the voxel weights kappa_n of Eq. (def_reg) in the oracle.

* the weighted regularizer against a brute-force sum over every neighbour pair
  (2-D, 8 neighbours, and 3-D, 26 neighbours) written here;
* kappa = 0 at one pixel removes every pair that contains it: R no longer
  depends on that pixel (a form that weighted a pair by kappa_n^2 would not);
* constant kappa = c scales R, its gradient and D_R by c^2;
* the gradient against central finite differences, and D_R majorizing R, with
  random kappa;
* resolution_kappa: uniform weights c give sqrt(c) on every pixel some ray
  meets and 0 elsewhere; on a tiny scan it equals the a_ij-weighted mean of w,
  summed here from the dense matrix; it lies between the smallest and the
  largest weight of the rays through the pixel; the helical projector gives
  sqrt(c) too;
* a relaxed OS-LALM solve with kappa reaches the KKT point of the weighted cost.
"""

import math

import numpy as np
import pytest

import synth
from oracle import regularizer as reg
from oracle import solver
from oracle.helical import HelicalProjector
from oracle.projector import FanProjector

KINDS = ["hyperbola", "fair", "quadratic"]


def _brute_value(x, kappa, beta, delta, kind):
    """sum over unordered neighbour pairs {n, m} of beta/||n - m|| kappa_n kappa_m phi(x_n - x_m)."""
    phi, _, _ = reg.potential(kind, delta)
    idx = list(np.ndindex(x.shape))
    tot = 0.0
    for a in idx:
        for b in idx:
            d = [bb - aa for aa, bb in zip(a, b)]
            if max(abs(c) for c in d) != 1 or tuple(d) <= tuple(-c for c in d):
                continue  # not a neighbour, or the pair's other orientation
            tot += beta / math.sqrt(sum(c * c for c in d)) * kappa[a] * kappa[b] * float(phi(x[a] - x[b]))
    return tot


@pytest.mark.parametrize("shape", [(4, 5), (3, 3, 4)])
@pytest.mark.parametrize("kind", KINDS)
def test_weighted_value_brute_force(shape, kind):
    rng = np.random.default_rng(11)
    x = rng.random(shape) * 0.05
    kappa = 0.5 + rng.random(shape)
    got = reg.value(x, 2.5, 0.01, kind, kappa)
    ref = _brute_value(x, kappa, 2.5, 0.01, kind)
    assert abs(got - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("shape", [(6, 7), (4, 5, 3)])
def test_zero_kappa_detaches_pixel(shape):
    rng = np.random.default_rng(5)
    x = rng.random(shape) * 0.05
    kappa = 0.5 + rng.random(shape)
    p = tuple(s // 2 for s in shape)
    kappa[p] = 0.0
    g = reg.gradient(x, 1.3, 0.01, "hyperbola", kappa)
    D = reg.curvature(x, 1.3, 0.01, "hyperbola", kappa)
    assert g[p] == 0.0 and D[p] == 0.0
    x2 = x.copy()
    x2[p] += 0.3
    assert abs(reg.value(x2, 1.3, 0.01, "hyperbola", kappa) - reg.value(x, 1.3, 0.01, "hyperbola", kappa)) < 1e-15
    # the neighbours of p still see their other pairs
    q = tuple(s - 1 if i == 0 else s for i, s in enumerate(p))
    assert g[q] != 0.0


@pytest.mark.parametrize("kind", KINDS)
def test_constant_kappa_scales_by_c_squared(kind):
    rng = np.random.default_rng(2)
    x = rng.random((6, 8)) * 0.05
    c = 1.7
    k = np.full(x.shape, c)
    assert abs(reg.value(x, 2.0, 0.01, kind, k) - c * c * reg.value(x, 2.0, 0.01, kind)) <= 1e-12 * abs(
        reg.value(x, 2.0, 0.01, kind, k))
    np.testing.assert_allclose(reg.gradient(x, 2.0, 0.01, kind, k), c * c * reg.gradient(x, 2.0, 0.01, kind),
                               rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(reg.curvature(x, 2.0, 0.01, kind, k), c * c * reg.curvature(x, 2.0, 0.01, kind),
                               rtol=1e-12)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("shape", [(7, 9), (4, 5, 6)])
def test_weighted_gradient_and_majorizer(kind, shape):
    rng = np.random.default_rng(7)
    delta = 0.05
    x = rng.random(shape) * 0.2
    kappa = 0.3 + rng.random(shape)
    g = reg.gradient(x, 3.0, delta, kind, kappa)
    eps = 1e-6
    for _ in range(12):
        j = tuple(int(rng.integers(0, s)) for s in shape)
        xp, xm = x.copy(), x.copy()
        xp[j] += eps
        xm[j] -= eps
        fd = (reg.value(xp, 3.0, delta, kind, kappa) - reg.value(xm, 3.0, delta, kind, kappa)) / (2 * eps)
        assert abs(fd - g[j]) <= 1e-6 * max(1.0, abs(g[j]))
    R0 = reg.value(x, 3.0, delta, kind, kappa)
    D = reg.curvature(x, 3.0, delta, kind, kappa)
    for _ in range(5):
        d = rng.normal(size=shape) * 0.1
        bound = R0 + np.sum(g * d) + 0.5 * np.sum(D * d * d)
        assert reg.value(x + d, 3.0, delta, kind, kappa) <= bound * (1 + 1e-12) + 1e-15


def _fan(nx=24, ns=24, na=36):
    # a narrow fan over a 60-degree arc: two image corners are met by no ray
    return synth.FanArcGeometry(nx=nx, ny=nx, dx=1.0, dy=1.0, ns=ns, ds=1.0, na=na, dso=60.0, dsd=100.0,
                                orbit_deg=60.0)


def test_resolution_kappa_uniform_weights():
    g = _fan()
    P = FanProjector(g)
    seen = P.back(np.ones((g.na, g.ns))) > 0
    assert seen.sum() > 0 and (~seen).sum() > 0
    k = solver.resolution_kappa(P, np.full((g.na, g.ns), 4.0))
    np.testing.assert_allclose(k[seen], 2.0, rtol=1e-13)
    assert np.all(k[~seen] == 0.0)


def test_resolution_kappa_matches_dense_mean():
    g = _fan(nx=8, ns=12, na=10)
    P = FanProjector(g)
    A = P.matrix()
    rng = np.random.default_rng(4)
    w = rng.uniform(10.0, 1000.0, size=(g.na, g.ns))
    k = solver.resolution_kappa(P, w).reshape(-1)
    wf = w.reshape(-1)
    for j in range(A.shape[1]):
        num = den = 0.0
        for i in range(A.shape[0]):
            num += A[i, j] * wf[i]
            den += A[i, j]
        if den > 0:
            assert abs(k[j] - math.sqrt(num / den)) <= 1e-12 * k[j]
            met = wf[A[:, j] > 0]
            assert met.min() * (1 - 1e-12) <= k[j] ** 2 <= met.max() * (1 + 1e-12)
        else:
            assert k[j] == 0.0


def test_resolution_kappa_helical_uniform():
    g = synth.HelicalConeGeometry(nx=10, ny=10, nz=4, dx=2.0, dy=2.0, dz=1.5, ns=24, ds=2.0, nt=4, dt=2.4, na=40,
                                  dso=200.0, dsd=350.0, pitch=0.8, orbit_deg=720.0)
    P = HelicalProjector(g)
    c = 9.0
    y1 = np.ones((g.na, g.nt, g.ns))
    seen = P.back(y1) > 0
    k = solver.resolution_kappa(P, c * y1)
    np.testing.assert_allclose(k[seen], 3.0, rtol=1e-13)
    assert np.all(k[~seen] == 0.0)


def test_weighted_solve_reaches_kkt_point():
    g = synth.FanArcGeometry(nx=20, ny=20, dx=1.0, dy=1.0, ns=40, ds=1.0, na=48, dso=100.0, dsd=180.0)
    E = [synth.Ellipse(0.0, 0.0, 7.0, 5.0, 0.2, 0.08), synth.Ellipse(2.0, 1.0, 2.0, 1.5, 0.0, 0.04)]
    y, w = synth.transmission_data(synth.fan_arc_line_integrals(E, g), 1e5, 5.0, 1)
    P = FanProjector(g)
    kappa = solver.resolution_kappa(P, w)
    unit = synth.configs.MU_WATER_PER_MM
    prob = solver.PWLSProblem(P, y, w, 400.0 / unit ** 2 / 1e5, 10 * unit / 1000.0, "hyperbola", kappa)
    x = np.zeros((g.ny, g.nx))
    for _ in range(3):
        x = solver.relaxed_os_lalm(prob, x, 1, 1.999, 300)
    r = solver.kkt_residual(prob, x)
    assert np.sqrt(np.mean(r ** 2)) < 1e-5 * np.abs(x).max()
    # kappa changes the solution (pixels with more weight are smoothed more)
    prob1 = solver.PWLSProblem(P, y, w, prob.beta * float(np.mean(kappa[kappa > 0] ** 2)), prob.delta)
    x1 = np.zeros_like(x)
    for _ in range(3):
        x1 = solver.relaxed_os_lalm(prob1, x1, 1, 1.999, 300)
    assert np.max(np.abs(x1 - x)) > 1e-3 * np.abs(x).max()
