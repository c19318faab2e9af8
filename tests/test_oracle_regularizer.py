"""Pins of the oracle regularizer (Sec. III, Eq. (def_reg)) and its Huber-curvature SQS.

* gradient against central finite differences of R;
* the quadratic potential against an explicitly assembled sum_i beta_i ||C_i x||^2 / 2
  (dense finite-difference matrices built here, not by the oracle);
* D_R(x) majorizes R around x (the majorization condition, Eq. (def_maj_diagonal));
* interior value of D_R for the quadratic potential: 4 sum_i beta_i;
* the potentials' small/large-argument limits.
"""

import math

import numpy as np
import pytest

from oracle import regularizer as reg

KINDS = ["hyperbola", "fair", "quadratic"]


def _dense_C(ny, nx, d):
    rows = []
    for iy in range(ny):
        for ix in range(nx):
            jx, jy = ix + d[0], iy + d[1]
            if 0 <= jx < nx and 0 <= jy < ny:
                r = np.zeros(ny * nx)
                r[iy * nx + ix] = 1.0
                r[jy * nx + jx] = -1.0
                rows.append(r)
    return np.array(rows)


@pytest.mark.parametrize("kind", KINDS)
def test_gradient_matches_finite_differences(kind):
    rng = np.random.default_rng(3)
    delta = 0.05
    x = rng.random((7, 9)) * 0.2
    g = reg.gradient(x, 3.0, delta, kind)
    eps = 1e-6
    for _ in range(12):
        j = (rng.integers(7), rng.integers(9))
        xp, xm = x.copy(), x.copy()
        xp[j] += eps
        xm[j] -= eps
        fd = (reg.value(xp, 3.0, delta, kind) - reg.value(xm, 3.0, delta, kind)) / (2 * eps)
        assert abs(fd - g[j]) <= 1e-6 * max(1.0, abs(g[j]))


def test_quadratic_matches_explicit_difference_matrices():
    rng = np.random.default_rng(4)
    ny, nx, beta = 6, 5, 2.5
    x = rng.standard_normal((ny, nx))
    dirs = [(1, 0), (0, 1), (1, 1), (1, -1)]
    w = [beta, beta, beta / math.sqrt(2), beta / math.sqrt(2)]
    H = sum(wi * _dense_C(ny, nx, d).T @ _dense_C(ny, nx, d) for wi, d in zip(w, dirs))
    xv = x.reshape(-1)
    assert abs(reg.value(x, beta, 1.0, "quadratic") - 0.5 * xv @ H @ xv) < 1e-12 * abs(xv @ H @ xv)
    np.testing.assert_allclose(reg.gradient(x, beta, 1.0, "quadratic").reshape(-1), H @ xv, atol=1e-12)
    # |C|'|C| 1 row sums: the SQS diagonal of the quadratic penalty
    absH = sum(wi * np.abs(_dense_C(ny, nx, d)).T @ np.abs(_dense_C(ny, nx, d)) for wi, d in zip(w, dirs))
    np.testing.assert_allclose(reg.curvature(x, beta, 1.0, "quadratic").reshape(-1), absH.sum(1), atol=1e-12)
    # interior pixel: every direction contributes 2 pairs x 2 = 4 beta_i
    assert abs(reg.curvature(x, beta, 1.0, "quadratic")[3, 2] - 4 * sum(w)) < 1e-12


@pytest.mark.parametrize("kind", KINDS)
def test_huber_curvature_majorizes(kind):
    rng = np.random.default_rng(5)
    delta = 0.03
    for _ in range(20):
        x = rng.random((8, 8)) * 0.3
        d = rng.standard_normal((8, 8)) * rng.choice([0.001, 0.05, 0.5])
        R0 = reg.value(x, 1.7, delta, kind)
        g = reg.gradient(x, 1.7, delta, kind)
        D = reg.curvature(x, 1.7, delta, kind)
        surrogate = R0 + np.sum(g * d) + 0.5 * np.sum(D * d * d)
        assert reg.value(x + d, 1.7, delta, kind) <= surrogate * (1 + 1e-12) + 1e-15


def test_potential_limits():
    delta = 0.01
    for kind in ("hyperbola", "fair"):
        phi, dphi, omega = reg.potential(kind, delta)
        t = np.array([1e-6])
        assert abs(phi(t)[0] - 0.5 * t[0] ** 2) < 1e-3 * 0.5 * t[0] ** 2  # quadratic near 0
        assert abs(omega(t)[0] - 1.0) < 1e-3
        T = np.array([1e3 * delta])
        assert abs(dphi(T)[0] - delta) < 2e-3 * delta  # slope -> delta for |t| >> delta
    phi, dphi, omega = reg.potential("hyperbola", delta)
    assert abs(phi(np.array([delta]))[0] - delta ** 2 * (math.sqrt(2) - 1)) < 1e-18
    phi, dphi, omega = reg.potential("fair", delta)
    assert abs(phi(np.array([delta]))[0] - delta ** 2 * (1 - math.log(2))) < 1e-18


@pytest.mark.parametrize("kind", ["hyperbola", "fair"])
def test_max_curvature_majorizes(kind):
    """phi''(0) = 1 bounds the curvature of both potentials, so 2 beta_i per pair majorizes R."""
    rng = np.random.default_rng(6)
    delta = 0.03
    for _ in range(20):
        x = rng.random((8, 8)) * 0.3
        d = rng.standard_normal((8, 8)) * rng.choice([0.001, 0.05, 0.5])
        R0 = reg.value(x, 1.7, delta, kind)
        g = reg.gradient(x, 1.7, delta, kind)
        D = reg.curvature(x, 1.7, delta, "quadratic")
        assert reg.value(x + d, 1.7, delta, kind) <= R0 + np.sum(g * d) + 0.5 * np.sum(D * d * d) + 1e-12
