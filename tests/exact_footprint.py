"""Brute-force reference footprints for pinning the SF projector.

Exact chord length of a ray through an axis-aligned rectangle (slab
intersection), integrated over a detector cell's fan-angle interval by
piecewise Gauss-Legendre quadrature between the rectangle's corner angles
(where the chord is smooth).  Written independently of the oracle's SF code.
"""

from __future__ import annotations

import math

import numpy as np


def chord_rect(sx, sy, dxr, dyr, x0, x1, y0, y1):
    """Length of {S + t d, t >= 0} inside [x0,x1]x[y0,y1]; d must be unit length."""
    tmin, tmax = 0.0, math.inf
    for s, d, lo, hi in ((sx, dxr, x0, x1), (sy, dyr, y0, y1)):
        if abs(d) < 1e-300:
            if s < lo or s > hi:
                return 0.0
            continue
        a, b = (lo - s) / d, (hi - s) / d
        if a > b:
            a, b = b, a
        tmin, tmax = max(tmin, a), min(tmax, b)
    return max(0.0, tmax - tmin)


def fan_angle(geom, beta, px, py):
    cb, sb = math.cos(beta), math.sin(beta)
    return math.atan2(-px * sb + py * cb, geom.dso + px * cb + py * sb)


def exact_cell_weight(geom, v, s, ix, iy, n_gauss=24):
    """(1/dgamma) * integral over cell s of the exact chord of pixel (ix, iy), view v."""
    beta = geom.betas()[v]
    cb, sb = math.cos(beta), math.sin(beta)
    Sx, Sy = -geom.dso * cb, -geom.dso * sb
    xc = (ix - (geom.nx - 1) / 2.0 + geom.offset_x) * geom.dx
    yc = (iy - (geom.ny - 1) / 2.0 + geom.offset_y) * geom.dy
    x0, x1 = xc - geom.dx / 2, xc + geom.dx / 2
    y0, y1 = yc - geom.dy / 2, yc + geom.dy / 2
    g_s = geom.gammas()[s]
    lo, hi = g_s - geom.dgamma / 2, g_s + geom.dgamma / 2
    corners = sorted(fan_angle(geom, beta, px, py) for px in (x0, x1) for py in (y0, y1))
    bps = [lo] + [c for c in corners if lo < c < hi] + [hi]
    xg, wg = np.polynomial.legendre.leggauss(n_gauss)
    total = 0.0
    for a, b in zip(bps[:-1], bps[1:]):
        for xi, wi in zip(xg, wg):
            gam = 0.5 * (a + b) + 0.5 * (b - a) * xi
            dxr = math.cos(gam) * cb - math.sin(gam) * sb
            dyr = math.cos(gam) * sb + math.sin(gam) * cb
            total += 0.5 * (b - a) * wi * chord_rect(Sx, Sy, dxr, dyr, x0, x1, y0, y1)
    return total / geom.dgamma


def exact_box_path(geom, v, s, n_gauss=24):
    """(1/dgamma) * integral over cell s of the chord through the whole image rectangle."""
    beta = geom.betas()[v]
    cb, sb = math.cos(beta), math.sin(beta)
    Sx, Sy = -geom.dso * cb, -geom.dso * sb
    hx = geom.nx * geom.dx / 2.0
    hy = geom.ny * geom.dy / 2.0
    ox, oy = geom.offset_x * geom.dx, geom.offset_y * geom.dy
    x0, x1, y0, y1 = ox - hx, ox + hx, oy - hy, oy + hy
    g_s = geom.gammas()[s]
    lo, hi = g_s - geom.dgamma / 2, g_s + geom.dgamma / 2
    corners = sorted(fan_angle(geom, beta, px, py) for px in (x0, x1) for py in (y0, y1))
    bps = [lo] + [c for c in corners if lo < c < hi] + [hi]
    xg, wg = np.polynomial.legendre.leggauss(n_gauss)
    total = 0.0
    for a, b in zip(bps[:-1], bps[1:]):
        for xi, wi in zip(xg, wg):
            gam = 0.5 * (a + b) + 0.5 * (b - a) * xi
            dxr = math.cos(gam) * cb - math.sin(gam) * sb
            dyr = math.cos(gam) * sb + math.sin(gam) * cb
            total += 0.5 * (b - a) * wi * chord_rect(Sx, Sy, dxr, dyr, x0, x1, y0, y1)
    return total / geom.dgamma
