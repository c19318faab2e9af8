"""Edge-preserving regularizer R, its gradient and its Huber-curvature SQS diagonal.

ORACLE -- test infrastructure only.

R(x) = sum_i beta_i sum_n kappa_n kappa_{n+s_i} phi([C_i x]_n)      (Sec. III, Eq. (def_reg))

with [C_i x]_n = x_n - x_{n+s_i}, counted for pairs whose both pixels lie in
the image, kappa_n the voxel-dependent weights (``kappa=None`` reads as
kappa = 1; ``resolution_kappa`` in oracle.solver gives the resolution-
uniformity choice), and beta_i = beta / ||s_i|| with ||s_i|| in index units
(axis neighbours beta, face diagonals beta/sqrt(2), body diagonals
beta/sqrt(3)).  In 2-D the four directions (1,0), (0,1), (1,1), (1,-1) cover
all 8 neighbours; in 3-D thirteen directions cover all 26 (the paper's 3-D
experiments use the 26 neighbours).  Offsets are (step in ix, step in iy[, step in iz])
and arrays are [iy][ix] or [iz][iy][ix].

The SQS diagonal uses Huber's curvature omega(t) = phi'(t)/t (Sec. III-A: the
iteration-dependent curvature used "for faster convergence"):

D_R(x) = |C|' diag(beta_i kappa_n kappa_{n+s_i} omega([C_i x]_n)) |C| 1, i.e.
each pair adds 2 beta_i kappa_n kappa_{n+s_i} omega(t) to both of its pixels
(|C_i| 1 = 2).
"""

from __future__ import annotations

import math

import numpy as np

DIRECTIONS_2D = ((1, 0), (0, 1), (1, 1), (1, -1))  # (step in ix, step in iy)
# one offset of each +-pair of the 26 neighbours: the first nonzero step is positive
DIRECTIONS_3D = tuple(d for d in ((i, j, k) for k in (-1, 0, 1) for j in (-1, 0, 1) for i in (-1, 0, 1))
                      if d != (0, 0, 0) and next(c for c in d if c != 0) > 0)


def directions(ndim: int):
    return DIRECTIONS_2D if ndim == 2 else DIRECTIONS_3D


def potential(kind: str, delta: float):
    """(phi, phi', omega = phi'(t)/t) for the hyperbola, Fair or quadratic potential."""
    if kind == "hyperbola":  # delta^2 (sqrt(1 + (t/delta)^2) - 1)
        phi = lambda t: delta * delta * (np.sqrt(1.0 + (t / delta) ** 2) - 1.0)  # noqa: E731
        dphi = lambda t: t / np.sqrt(1.0 + (t / delta) ** 2)  # noqa: E731
        omega = lambda t: 1.0 / np.sqrt(1.0 + (t / delta) ** 2)  # noqa: E731
    elif kind == "fair":  # delta^2 (|t/delta| - log(1 + |t/delta|)), Sec. IV-A
        phi = lambda t: delta * delta * (np.abs(t / delta) - np.log1p(np.abs(t / delta)))  # noqa: E731
        dphi = lambda t: t / (1.0 + np.abs(t) / delta)  # noqa: E731
        omega = lambda t: 1.0 / (1.0 + np.abs(t) / delta)  # noqa: E731
    elif kind == "quadratic":  # t^2 / 2
        phi = lambda t: 0.5 * t * t  # noqa: E731
        dphi = lambda t: np.asarray(t, dtype=np.float64) * 1.0  # noqa: E731
        omega = lambda t: np.ones_like(np.asarray(t, dtype=np.float64))  # noqa: E731
    else:
        raise ValueError(kind)
    return phi, dphi, omega


def direction_weights(beta: float, dirs=DIRECTIONS_2D):
    return [beta / math.sqrt(sum(c * c for c in d)) for d in dirs]


def _pair_slices(shape, d):
    """Slices (a, b) so that x[a] and x[b] are the pairs n, n + s (both inside the array).

    ``d`` lists steps along (ix, iy[, iz]); ``shape`` is (ny, nx) or (nz, ny, nx).
    """

    def one(step, n):
        return (slice(0, n - step), slice(step, n)) if step >= 0 else (slice(-step, n), slice(0, n + step))

    axes = [one(step, n) for step, n in zip(d, shape[::-1])]  # along x, y[, z]
    a = tuple(p[0] for p in axes[::-1])
    b = tuple(p[1] for p in axes[::-1])
    return a, b


def _pair_weight(kappa, a, b):
    """kappa_n kappa_{n+s_i} of each pair (1 without kappa)."""
    return 1.0 if kappa is None else kappa[a] * kappa[b]


def value(x: np.ndarray, beta: float, delta: float, kind: str, kappa: np.ndarray | None = None) -> float:
    phi, _, _ = potential(kind, delta)
    dirs = directions(x.ndim)
    tot = 0.0
    for d, bi in zip(dirs, direction_weights(beta, dirs)):
        a, b = _pair_slices(x.shape, d)
        tot += bi * float(np.sum(_pair_weight(kappa, a, b) * phi(x[a] - x[b])))
    return tot


def gradient(x: np.ndarray, beta: float, delta: float, kind: str, kappa: np.ndarray | None = None) -> np.ndarray:
    _, dphi, _ = potential(kind, delta)
    dirs = directions(x.ndim)
    g = np.zeros_like(x, dtype=np.float64)
    for d, bi in zip(dirs, direction_weights(beta, dirs)):
        a, b = _pair_slices(x.shape, d)
        f = bi * _pair_weight(kappa, a, b) * dphi(x[a] - x[b])
        g[a] += f
        g[b] -= f
    return g


def curvature(x: np.ndarray, beta: float, delta: float, kind: str, kappa: np.ndarray | None = None) -> np.ndarray:
    """Huber-curvature SQS diagonal D_R(x)."""
    _, _, omega = potential(kind, delta)
    dirs = directions(x.ndim)
    D = np.zeros_like(x, dtype=np.float64)
    for d, bi in zip(dirs, direction_weights(beta, dirs)):
        a, b = _pair_slices(x.shape, d)
        c = 2.0 * bi * _pair_weight(kappa, a, b) * omega(x[a] - x[b])
        D[a] += c
        D[b] += c
    return D
