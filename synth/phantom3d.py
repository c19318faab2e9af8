"""3-D phantoms (ellipsoids and z-limited elliptic cylinders) and their
closed-form helical cone-beam line integrals.

The line integral of a uniform solid along a line is its value times the
length of the line inside it.  For an ellipsoid that length comes from the
roots of a quadratic in the line parameter; for an elliptic cylinder
capped by two planes z = z0, z = z1 it is the overlap of the quadratic's
root interval (transaxial ellipse) with the interval where z0 <= z <= z1.
Sinograms built from these closed forms never go through a voxel-basis
system matrix.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

from .configs import HelicalConeGeometry
from .rng import philox


@dataclasses.dataclass(frozen=True)
class Ellipsoid:
    cx: float
    cy: float
    cz: float
    a: float  # semi-axis along its own x axis (mm)
    b: float  # along its own y axis
    c: float  # along z
    theta: float  # rotation about z (rad)
    value: float  # additive attenuation (1/mm)


@dataclasses.dataclass(frozen=True)
class EllipticCylinder:
    cx: float
    cy: float
    a: float
    b: float
    theta: float
    z0: float  # caps (mm), z0 < z1
    z1: float
    value: float


def _frame(sx, sy, dxr, dyr, cx, cy, theta):
    c, s = math.cos(theta), math.sin(theta)
    px = c * (sx - cx) + s * (sy - cy)
    py = -s * (sx - cx) + c * (sy - cy)
    qx = c * dxr + s * dyr
    qy = -s * dxr + c * dyr
    return px, py, qx, qy


def chord_lengths(solids, sx, sy, sz, dxr, dyr, dzr) -> np.ndarray:
    """Sum over solids of value x length of the lines S + t d (d unit) inside them (broadcast arrays)."""
    shape = np.broadcast(sx, sy, sz, dxr, dyr, dzr).shape
    total = np.zeros(shape, dtype=np.float64)
    for e in solids:
        px, py, qx, qy = _frame(sx, sy, dxr, dyr, e.cx, e.cy, e.theta)
        if isinstance(e, Ellipsoid):
            pz, qz = sz - e.cz, dzr
            A = (qx / e.a) ** 2 + (qy / e.b) ** 2 + (qz / e.c) ** 2
            B = 2.0 * (px * qx / e.a ** 2 + py * qy / e.b ** 2 + pz * qz / e.c ** 2)
            C = (px / e.a) ** 2 + (py / e.b) ** 2 + (pz / e.c) ** 2 - 1.0
            disc = B * B - 4.0 * A * C
            total += e.value * np.sqrt(np.maximum(disc, 0.0)) / A
        else:
            A = (qx / e.a) ** 2 + (qy / e.b) ** 2
            B = 2.0 * (px * qx / e.a ** 2 + py * qy / e.b ** 2)
            C = (px / e.a) ** 2 + (py / e.b) ** 2 - 1.0
            disc = B * B - 4.0 * A * C
            ok = (disc > 0.0) & (A > 0.0)
            r = np.sqrt(np.maximum(disc, 0.0))
            Asafe = np.where(A > 0.0, A, 1.0)
            t_lo = np.where(ok, (-B - r) / (2.0 * Asafe), 0.0)
            t_hi = np.where(ok, (-B + r) / (2.0 * Asafe), 0.0)
            # slab z0 <= sz + t dz <= z1
            dz_safe = np.where(np.abs(dzr) > 1e-300, dzr, 1.0)
            ta = (e.z0 - sz) / dz_safe
            tb = (e.z1 - sz) / dz_safe
            inside_flat = (sz >= e.z0) & (sz <= e.z1)
            s_lo = np.where(np.abs(dzr) > 1e-300, np.minimum(ta, tb), np.where(inside_flat, -np.inf, np.inf))
            s_hi = np.where(np.abs(dzr) > 1e-300, np.maximum(ta, tb), np.where(inside_flat, np.inf, -np.inf))
            total += e.value * np.maximum(np.minimum(t_hi, s_hi) - np.maximum(t_lo, s_lo), 0.0) * ok
    return total


def _ray_dirs(g: HelicalConeGeometry, beta, gam, h):
    """Unit direction of the ray from the source to the detector point at fan angle gam, height h."""
    phi = beta + gam
    dxr, dyr = g.dsd * np.cos(phi), g.dsd * np.sin(phi)
    n = np.sqrt(dxr * dxr + dyr * dyr + h * h)
    return dxr / n, dyr / n, h / n


def _bounding_sphere(e):
    if isinstance(e, Ellipsoid):
        return e.cx, e.cy, e.cz, max(e.a, e.b, e.c)
    return e.cx, e.cy, 0.5 * (e.z0 + e.z1), math.hypot(max(e.a, e.b), 0.5 * (e.z1 - e.z0))


def _detector_window(g: HelicalConeGeometry, beta, sx, sy, sz, sphere):
    """Cells [s0, s1) and rows [t0, t1) that rays meeting the sphere can reach (padded by one)."""
    px, py, pz, r = sphere
    dxy = math.hypot(px - sx, py - sy)
    if dxy <= r * 1.0001:
        return 0, g.ns, 0, g.nt
    phc = math.atan2(py - sy, px - sx) - beta
    phc = (phc + math.pi) % (2.0 * math.pi) - math.pi
    half = math.asin(r / dxy)
    c0 = (g.ns - 1) / 2.0 - g.offset_s
    s0 = int(math.floor((phc - half) / g.dgamma + c0)) - 1
    s1 = int(math.ceil((phc + half) / g.dgamma + c0)) + 2
    hs = [(z - sz) * g.dsd / L for z in (pz - r, pz + r) for L in (dxy - r, dxy + r)]
    r0 = (g.nt - 1) / 2.0 - g.offset_t
    t0 = int(math.floor(min(hs) / g.dt + r0)) - 1
    t1 = int(math.ceil(max(hs) / g.dt + r0)) + 2
    return max(s0, 0), min(s1, g.ns), max(t0, 0), min(t1, g.nt)


def helical_line_integrals(solids, g: HelicalConeGeometry, n_sub: int = 2, views=None) -> np.ndarray:
    """Cell-averaged analytic line integrals ``[nviews][nt][ns]``.

    Each detector cell averages ``n_sub x n_sub`` rays placed at the
    Gauss-Legendre nodes of its fan-angle and height extents.  Each solid is
    evaluated only on the detector window its bounding sphere projects to.
    """
    views = np.arange(g.na) if views is None else np.asarray(views)
    betas = g.betas()[views]
    gam = g.gammas()
    hts = g.row_heights()
    xg, wg = np.polynomial.legendre.leggauss(n_sub)
    spheres = [_bounding_sphere(e) for e in solids]
    out = np.zeros((len(views), g.nt, g.ns), dtype=np.float64)
    for vi, b in enumerate(betas):
        sx, sy, sz = -g.dso * math.cos(b), -g.dso * math.sin(b), g.source_z(b)
        acc = out[vi]
        for e, sph in zip(solids, spheres):
            s0, s1, t0, t1 = _detector_window(g, b, sx, sy, sz, sph)
            if s0 >= s1 or t0 >= t1:
                continue
            for xa, wa in zip(xg, wg):
                ga = (gam[s0:s1] + 0.5 * g.dgamma * xa)[None, :]
                for xb, wb in zip(xg, wg):
                    hb = (hts[t0:t1] + 0.5 * g.dt * xb)[:, None]
                    dxr, dyr, dzr = _ray_dirs(g, b, ga, hb)
                    acc[t0:t1, s0:s1] += 0.25 * wa * wb * chord_lengths([e], sx, sy, sz, dxr, dyr, dzr)
    return out


def helical_line_integrals_sampled(solids, g: HelicalConeGeometry, ray_view, ray_row, ray_cell,
                                   n_sub: int = 2) -> np.ndarray:
    """Same as :func:`helical_line_integrals` for an explicit list of (view, row, cell) rays."""
    b = g.betas()[np.asarray(ray_view)]
    gam = g.gammas()[np.asarray(ray_cell)]
    hts = g.row_heights()[np.asarray(ray_row)]
    sx, sy = -g.dso * np.cos(b), -g.dso * np.sin(b)
    sz = np.array([g.source_z(bb) for bb in b])
    xg, wg = np.polynomial.legendre.leggauss(n_sub)
    acc = np.zeros(len(b))
    for xa, wa in zip(xg, wg):
        for xb, wb in zip(xg, wg):
            dxr, dyr, dzr = _ray_dirs(g, b, gam + 0.5 * g.dgamma * xa, hts + 0.5 * g.dt * xb)
            acc += 0.25 * wa * wb * chord_lengths(solids, sx, sy, sz, dxr, dyr, dzr)
    return acc


def rasterize_solids(solids, g: HelicalConeGeometry, oversample: int = 4, oversample_z: int = 4) -> np.ndarray:
    """Voxel-average volume ``[nz][ny][nx]`` by ``oversample^2 * oversample_z`` sub-samples per voxel."""
    k, kz = oversample, oversample_z
    sub = (np.arange(k) + 0.5) / k - 0.5
    subz = (np.arange(kz) + 0.5) / kz - 0.5
    xc = (np.arange(g.nx) - (g.nx - 1) / 2.0 + g.offset_x) * g.dx
    yc = (np.arange(g.ny) - (g.ny - 1) / 2.0 + g.offset_y) * g.dy
    zc = (np.arange(g.nz) - (g.nz - 1) / 2.0 + g.offset_z) * g.dz
    vol = np.zeros((g.nz, g.ny, g.nx))
    for qz in subz:
        Z = (zc + qz * g.dz)[:, None, None]
        for qy in sub:
            Y = (yc + qy * g.dy)[None, :, None]
            for qx in sub:
                X = (xc + qx * g.dx)[None, None, :]
                for e in solids:
                    c, s = math.cos(e.theta), math.sin(e.theta)
                    u = c * (X - e.cx) + s * (Y - e.cy)
                    v = -s * (X - e.cx) + c * (Y - e.cy)
                    if isinstance(e, Ellipsoid):
                        inside = (u / e.a) ** 2 + (v / e.b) ** 2 + ((Z - e.cz) / e.c) ** 2 <= 1.0
                    else:
                        inside = ((u / e.a) ** 2 + (v / e.b) ** 2 <= 1.0) & (Z >= e.z0) & (Z <= e.z1)
                    vol += e.value * inside
    return vol / (k * k * kz)


def random_solids(seed: int, r_max: float, z_half: float, mu_max: float = 0.02) -> list:
    """A body cylinder (radius ~r_max, caps at +-z_half) with eight non-overlapping ellipsoid inserts."""
    rng = philox(seed, stream=404)
    mu_b = rng.uniform(0.012, 0.018)
    a_b, b_b = rng.uniform(0.85, 0.97) * r_max, rng.uniform(0.7, 0.9) * r_max
    th_b = rng.uniform(0, math.pi)
    out: list = [EllipticCylinder(0.0, 0.0, a_b, b_b, th_b, -z_half, z_half, mu_b)]
    placed: list[tuple[float, float, float, float, float]] = []
    tries = 0
    while len(out) < 9 and tries < 20000:
        tries += 1
        r = rng.uniform(0.08, 0.25) * r_max
        u, v = rng.uniform(-1, 1, size=2)
        if u * u + v * v > 1.0:
            continue
        px, py = u * (a_b - r - 1.0), v * (b_b - r - 1.0)
        if (px / max(a_b - r - 1.0, 1e-3)) ** 2 + (py / max(b_b - r - 1.0, 1e-3)) ** 2 > 1.0:
            continue
        c, s = math.cos(th_b), math.sin(th_b)
        cx, cy = c * px - s * py, s * px + c * py
        rz = rng.uniform(0.3, 0.8) * z_half
        cz = rng.uniform(-(z_half - rz), z_half - rz)
        if any(math.hypot(cx - qx, cy - qy) < r + qr + 1.0 and abs(cz - qz) < rz + qrz + 0.5
               for qx, qy, qr, qz, qrz in placed):
            continue
        placed.append((cx, cy, r, cz, rz))
        out.append(Ellipsoid(cx, cy, cz, r, r * rng.uniform(0.6, 1.0), rz, rng.uniform(0, math.pi),
                             rng.uniform(-mu_b, mu_max - mu_b)))
    return out


def anthropomorphic_solids(seed: int, z_half: float, scale: float = 1.0) -> list:
    """Chest-like 3-D phantom with values in [0, 0.025]/mm: body, lungs and spine as capped elliptic
    cylinders (caps at +-z_half), heart, sternum and lesions as ellipsoids inside them."""
    rng = philox(seed, stream=505)
    j = lambda lo, hi: rng.uniform(lo, hi)  # noqa: E731
    zh = z_half
    body_mu = 0.019
    S: list = [EllipticCylinder(0.0, 0.0, 195 * scale * j(0.97, 1.0), 145 * scale * j(0.97, 1.0), j(-0.03, 0.03),
                                -zh, zh, body_mu)]
    S.append(EllipticCylinder(-92 * scale, 12 * scale, 58 * scale * j(0.95, 1.05), 88 * scale * j(0.95, 1.05),
                              j(-0.2, -0.05), -zh, zh, 0.004 - body_mu))
    S.append(EllipticCylinder(92 * scale, 12 * scale, 58 * scale * j(0.95, 1.05), 88 * scale * j(0.95, 1.05),
                              j(0.05, 0.2), -zh, zh, 0.004 - body_mu))
    S.append(Ellipsoid(5 * scale, 30 * scale, j(-0.3, 0.3) * zh, 28 * scale * j(0.95, 1.05), 24 * scale * j(0.95, 1.05),
                       0.9 * zh, j(0, math.pi), 0.021 - body_mu))
    S.append(EllipticCylinder(0.0, -100 * scale, 17 * scale * j(0.95, 1.05), 15 * scale * j(0.95, 1.05), 0.0,
                              -zh, zh, 0.025 - body_mu))
    S.append(Ellipsoid(0.0, 118 * scale, 0.0, 10 * scale, 5 * scale, 0.8 * zh, 0.0, 0.024 - body_mu))
    n = 0
    tries = 0
    placed: list[tuple[float, float, float]] = []
    while n < 12 and tries < 20000:
        tries += 1
        r = rng.uniform(2.0, 9.0) * scale
        rz = min(r, 0.45 * zh)
        cz = rng.uniform(-(zh - rz - 0.5), zh - rz - 0.5)
        if n < 6:  # lung nodules
            side = -1.0 if n % 2 == 0 else 1.0
            lung = S[1] if side < 0 else S[2]
            cx = lung.cx + rng.uniform(-40, 40) * scale
            cy = lung.cy + rng.uniform(-65, 65) * scale
            if ((cx - lung.cx) / (lung.a - r - 2)) ** 2 + ((cy - lung.cy) / (lung.b - r - 2)) ** 2 > 1.0:
                continue
            val = rng.uniform(0.008, 0.012)
        else:  # soft-tissue lesions of +-30..150 HU, away from the other inner structures
            cx, cy = rng.uniform(-170, 170) * scale, rng.uniform(-125, 125) * scale
            b0 = S[0]
            if (cx / (b0.a - r - 4)) ** 2 + (cy / (b0.b - r - 4)) ** 2 > 1.0:
                continue
            if any(((cx - e.cx) / (e.a + r + 1)) ** 2 + ((cy - e.cy) / (e.b + r + 1)) ** 2 <= 1.0 for e in S[1:6]):
                continue
            val = rng.choice([-1.0, 1.0]) * rng.uniform(0.0006, 0.003)
        if any(math.hypot(cx - qx, cy - qy) < r + qr + 1.0 for qx, qy, qr in placed):
            continue
        placed.append((cx, cy, r))
        S.append(Ellipsoid(cx, cy, cz, r, r * rng.uniform(0.6, 1.0), rz, rng.uniform(0, math.pi), val))
        n += 1
    return S
