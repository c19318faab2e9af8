"""Ellipse phantoms and their closed-form fan-beam line integrals.

The line integral of a uniform ellipse along a line is the chord length times
the ellipse's value; the chord comes from the roots of a quadratic in the
line parameter.  Sinograms built from these closed forms do not go through
any discretised system matrix, so reconstructing them with a pixel-basis
projector commits no "inverse crime".
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

from .configs import FanArcGeometry
from .rng import philox


@dataclasses.dataclass(frozen=True)
class Ellipse:
    cx: float  # centre (mm)
    cy: float
    a: float  # semi-axis along the ellipse's own x axis (mm)
    b: float  # semi-axis along the ellipse's own y axis (mm)
    theta: float  # rotation (rad), counter-clockwise
    value: float  # additive attenuation (1/mm)


def random_ellipses_cfg1(seed: int, r_max: float = 60.0, mu_max: float = 0.02) -> list[Ellipse]:
    """Ten seeded ellipses inside a disk of radius ``r_max``, values summing to [0, mu_max].

    One body ellipse plus nine non-overlapping inserts strictly inside it, so
    every point's total attenuation stays in [0, mu_max].
    """
    rng = philox(seed, stream=101)
    mu_b = rng.uniform(0.012, 0.018)
    a_b = rng.uniform(0.85, 0.97) * r_max
    b_b = rng.uniform(0.70, 0.90) * r_max
    th_b = rng.uniform(0, math.pi)
    out = [Ellipse(0.0, 0.0, a_b, b_b, th_b, mu_b)]
    placed: list[tuple[float, float, float]] = []
    tries = 0
    while len(out) < 10 and tries < 10000:
        tries += 1
        ra = rng.uniform(3.0, 14.0)
        rb = rng.uniform(0.4, 1.0) * ra
        # centre inside the body (in its frame) with a margin of ra
        u, v = rng.uniform(-1, 1, size=2)
        if u * u + v * v > 1.0:
            continue
        px, py = u * (a_b - ra - 1.0), v * (b_b - ra - 1.0)
        if px * px / max(a_b - ra - 1.0, 1e-3) ** 2 + py * py / max(b_b - ra - 1.0, 1e-3) ** 2 > 1.0:
            continue
        c, s = math.cos(th_b), math.sin(th_b)
        cx, cy = c * px - s * py, s * px + c * py
        if any(math.hypot(cx - qx, cy - qy) < ra + qr + 1.0 for qx, qy, qr in placed):
            continue
        placed.append((cx, cy, ra))
        contrast = rng.uniform(-mu_b, mu_max - mu_b)
        out.append(Ellipse(cx, cy, ra, rb, rng.uniform(0, math.pi), contrast))
    return out


def anthropomorphic_ellipses(seed: int, scale: float = 1.0) -> list[Ellipse]:
    """Chest-like ellipse phantom with values in [0, 0.025]/mm (body, lungs, heart, spine, lesions).

    Shapes follow a transaxial chest slice at roughly the size of the
    paper's XCAT and chest reconstructions (about 400 x 300 mm body); every
    inner structure sits inside the body and no two inner structures overlap.
    """
    rng = philox(seed, stream=202)
    j = lambda lo, hi: rng.uniform(lo, hi)  # noqa: E731
    body_mu = 0.019
    E: list[Ellipse] = [Ellipse(0.0, 0.0, 195 * scale * j(0.97, 1.0), 145 * scale * j(0.97, 1.0), j(-0.03, 0.03), body_mu)]
    # lungs (value ~0.004), heart (0.021), spine (0.025), sternum (0.024)
    E.append(Ellipse(-92 * scale, 12 * scale, 58 * scale * j(0.95, 1.05), 88 * scale * j(0.95, 1.05), j(-0.2, -0.05), 0.004 - body_mu))
    E.append(Ellipse(92 * scale, 12 * scale, 58 * scale * j(0.95, 1.05), 88 * scale * j(0.95, 1.05), j(0.05, 0.2), 0.004 - body_mu))
    E.append(Ellipse(5 * scale, 30 * scale, 28 * scale * j(0.95, 1.05), 24 * scale * j(0.95, 1.05), j(0, math.pi), 0.021 - body_mu))
    E.append(Ellipse(0.0, -100 * scale, 17 * scale * j(0.95, 1.05), 15 * scale * j(0.95, 1.05), 0.0, 0.025 - body_mu))
    E.append(Ellipse(0.0, 118 * scale, 10 * scale, 5 * scale, 0.0, 0.024 - body_mu))
    placed = [(e.cx, e.cy, max(e.a, e.b)) for e in E[1:]]
    # small lesions: inside the lungs (denser than lung) and in soft tissue
    n_lesion = 0
    tries = 0
    while n_lesion < 12 and tries < 20000:
        tries += 1
        r = rng.uniform(2.0, 9.0) * scale
        if n_lesion < 6:  # lung nodules
            side = -1.0 if n_lesion % 2 == 0 else 1.0
            cx = side * 92 * scale + rng.uniform(-40, 40) * scale
            cy = 12 * scale + rng.uniform(-65, 65) * scale
            lung = E[1] if side < 0 else E[2]
            if ((cx - lung.cx) / (lung.a - r - 2)) ** 2 + ((cy - lung.cy) / (lung.b - r - 2)) ** 2 > 1.0:
                continue
            if any(math.hypot(cx - qx, cy - qy) < r + qr + 1.0 for qx, qy, qr in placed[5:]):
                continue
            E.append(Ellipse(cx, cy, r, r * rng.uniform(0.6, 1.0), rng.uniform(0, math.pi), rng.uniform(0.008, 0.012)))
        else:  # soft-tissue lesions of +-30..150 HU
            cx = rng.uniform(-170, 170) * scale
            cy = rng.uniform(-125, 125) * scale
            b0 = E[0]
            if (cx / (b0.a - r - 4)) ** 2 + (cy / (b0.b - r - 4)) ** 2 > 1.0:
                continue
            if any(math.hypot(cx - qx, cy - qy) < r + qr + 1.0 for qx, qy, qr in placed):
                continue
            E.append(Ellipse(cx, cy, r, r * rng.uniform(0.6, 1.0), rng.uniform(0, math.pi),
                             rng.choice([-1.0, 1.0]) * rng.uniform(0.0006, 0.003)))
        placed.append((cx, cy, r))
        n_lesion += 1
    return E


def rasterize_ellipses(ellipses: list[Ellipse], nx: int, ny: int, dx: float, dy: float,
                       offset_x: float = 0.0, offset_y: float = 0.0, oversample: int = 8) -> np.ndarray:
    """Pixel-average image ``[ny][nx]`` of the phantom, by ``oversample**2`` sub-samples per pixel."""
    k = oversample
    sub = (np.arange(k) + 0.5) / k - 0.5
    xc = (np.arange(nx) - (nx - 1) / 2.0 + offset_x) * dx
    yc = (np.arange(ny) - (ny - 1) / 2.0 + offset_y) * dy
    img = np.zeros((ny, nx), dtype=np.float64)
    for sy in sub:
        Y = (yc + sy * dy)[:, None]
        for sx in sub:
            X = (xc + sx * dx)[None, :]
            for e in ellipses:
                c, s = math.cos(e.theta), math.sin(e.theta)
                u = c * (X - e.cx) + s * (Y - e.cy)
                v = -s * (X - e.cx) + c * (Y - e.cy)
                img += e.value * ((u / e.a) ** 2 + (v / e.b) ** 2 <= 1.0)
    return img / (k * k)


def _chords(ellipses, sx, sy, dxr, dyr):
    """Sum over ellipses of value x chord length of lines S + t d (d unit), broadcast arrays."""
    total = np.zeros(np.broadcast(sx, dxr).shape, dtype=np.float64)
    for e in ellipses:
        c, s = math.cos(e.theta), math.sin(e.theta)
        px = c * (sx - e.cx) + s * (sy - e.cy)
        py = -s * (sx - e.cx) + c * (sy - e.cy)
        qx = c * dxr + s * dyr
        qy = -s * dxr + c * dyr
        A = (qx / e.a) ** 2 + (qy / e.b) ** 2
        B = 2.0 * (px * qx / e.a ** 2 + py * qy / e.b ** 2)
        C = (px / e.a) ** 2 + (py / e.b) ** 2 - 1.0
        disc = B * B - 4.0 * A * C
        total += e.value * np.sqrt(np.maximum(disc, 0.0)) / A
    return total


def fan_arc_line_integrals(ellipses: list[Ellipse], g: FanArcGeometry, n_gauss: int = 8,
                           views: np.ndarray | None = None) -> np.ndarray:
    """Bin-averaged analytic line integrals ``[nviews][ns]`` for a fan-arc scan.

    Each detector bin integrates over its angular width (a rectangular
    detector response), evaluated with ``n_gauss``-point Gauss-Legendre
    quadrature in the fan angle.
    """
    betas = g.betas() if views is None else g.betas()[np.asarray(views)]
    gam = g.gammas()
    xg, wg = np.polynomial.legendre.leggauss(n_gauss)
    out = np.zeros((len(betas), g.ns), dtype=np.float64)
    for vi, b in enumerate(betas):
        cb, sb = math.cos(b), math.sin(b)
        sx, sy = -g.dso * cb, -g.dso * sb
        gq = gam[:, None] + 0.5 * g.dgamma * xg[None, :]
        dxr = np.cos(gq) * cb - np.sin(gq) * sb
        dyr = np.cos(gq) * sb + np.sin(gq) * cb
        vals = _chords(ellipses, sx, sy, dxr, dyr)
        out[vi] = 0.5 * (vals * wg[None, :]).sum(axis=1)
    return out


def fan_arc_line_integrals_sampled(ellipses: list[Ellipse], g: FanArcGeometry, ray_view: np.ndarray,
                                   ray_bin: np.ndarray, n_gauss: int = 8) -> np.ndarray:
    """Same as :func:`fan_arc_line_integrals` for an explicit list of (view, bin) rays."""
    betas = g.betas()[np.asarray(ray_view)]
    gam = g.gammas()[np.asarray(ray_bin)]
    xg, wg = np.polynomial.legendre.leggauss(n_gauss)
    cb, sb = np.cos(betas)[:, None], np.sin(betas)[:, None]
    gq = gam[:, None] + 0.5 * g.dgamma * xg[None, :]
    dxr = np.cos(gq) * cb - np.sin(gq) * sb
    dyr = np.cos(gq) * sb + np.sin(gq) * cb
    vals = _chords(ellipses, -g.dso * cb, -g.dso * sb, dxr, dyr)
    return 0.5 * (vals * wg[None, :]).sum(axis=1)
