"""Filtered back-projection for an equiangular fan beam (initial image of Algorithm 1).

ORACLE -- test infrastructure only.

Algorithm 1 starts from "an initial (FBP) image" (Sec. III-A) without
specifying it; this is the textbook equiangular fan-beam FBP (Kak & Slaney,
"Principles of Computerized Tomographic Imaging", Ch. 3, fan beams with
equiangular rays) over a full 360-degree scan:

  1. pre-weight   p'(beta, gamma) = D cos(gamma) p(beta, gamma), D = source-to-isocentre;
  2. filter       q(beta, gamma_s) = dgamma sum_k p'(beta, gamma_k) g((s - k) dgamma), with the
                  band-limited kernel g(0) = 1/(8 dgamma^2), g(n dgamma) = 0 for even n != 0,
                  g(n dgamma) = -1 / (2 pi^2 sin^2(n dgamma)) for odd n
                  (optionally multiplied in frequency by a Hann window, applied here as the
                  spatial convolution with the kernel's Hann-apodised version);
  3. back-project f(x, y) = dbeta sum_views q(beta, gamma'(x, y)) / L(x, y, beta)^2, with
                  gamma' the fan angle of the point, L its distance from the source, and
                  q sampled at gamma' by linear interpolation (0 outside the detector).

For a helical scan (ssrb_sinogram, fbp_helical_ssrb) each slice is first rebinned to a 2-D fan
sinogram of one turn (single-slice rebinning), then reconstructed as above.
"""

from __future__ import annotations

import math

import numpy as np


def ramp_kernel(ns: int, dgamma: float, window: str = "ramp") -> np.ndarray:
    """Kernel values g(n dgamma) for n = -(ns-1) .. ns-1."""
    n = np.arange(-(ns - 1), ns)
    g = np.zeros(n.size, dtype=np.float64)
    g[n == 0] = 1.0 / (8.0 * dgamma * dgamma)
    odd = (n % 2) != 0
    g[odd] = -1.0 / (2.0 * math.pi ** 2 * np.sin(n[odd] * dgamma) ** 2)
    if window == "hann":
        # Hann apodisation of the ramp: convolve with the 3-tap kernel [1/4, 1/2, 1/4]
        gp = np.pad(g, 1)
        g = 0.25 * gp[:-2] + 0.5 * gp[1:-1] + 0.25 * gp[2:]
    elif window != "ramp":
        raise ValueError(window)
    return g


def fbp_fan_arc(geom, sino: np.ndarray, window: str = "ramp") -> np.ndarray:
    """FBP image [ny][nx] (same units as the line integrals per mm) from a full-scan sinogram [na][ns]."""
    g = geom
    dgamma = g.dgamma
    gam = g.gammas()
    betas = g.betas()
    dbeta = np.deg2rad(g.orbit_deg) / g.na
    pw = g.dso * np.cos(gam)[None, :] * np.asarray(sino, dtype=np.float64)
    ker = ramp_kernel(g.ns, dgamma, window)
    q = np.empty_like(pw)
    for v in range(g.na):
        q[v] = dgamma * np.convolve(pw[v], ker, mode="valid")  # length ns: sum_k p'[k] g[s-k]
    xc = (np.arange(g.nx) - (g.nx - 1) / 2.0 + g.offset_x) * g.dx
    yc = (np.arange(g.ny) - (g.ny - 1) / 2.0 + g.offset_y) * g.dy
    X, Y = np.meshgrid(xc, yc)
    img = np.zeros((g.ny, g.nx), dtype=np.float64)
    c0 = (g.ns - 1) / 2.0 - g.offset_s
    for v, b in enumerate(betas):
        cb, sb = math.cos(b), math.sin(b)
        tpar = g.dso + X * cb + Y * sb
        tperp = -X * sb + Y * cb
        L2 = tpar * tpar + tperp * tperp
        u = np.arctan2(tperp, tpar) / dgamma + c0
        i0 = np.floor(u).astype(np.int64)
        f = u - i0
        v0 = np.where((i0 >= 0) & (i0 < g.ns), q[v][np.clip(i0, 0, g.ns - 1)], 0.0)
        v1 = np.where((i0 + 1 >= 0) & (i0 + 1 < g.ns), q[v][np.clip(i0 + 1, 0, g.ns - 1)], 0.0)
        img += ((1.0 - f) * v0 + f * v1) / L2
    return img * dbeta


def ssrb_sinogram(geom, sino: np.ndarray, k: int):
    """Single-slice rebinning of a helical scan for slice k: (v0, p) with p [na_turn][ns] the 2-D
    fan-beam sinogram of the one-turn window of views v0 .. v0 + na_turn - 1.

    The paper starts Algorithm 1 from an FBP image (Sec. IV) but gives no helical FBP; this start image
    is the textbook single-slice rebinning (each view contributes the detector row where the slice's
    height at the isocentre projects, interpolated linearly between rows, times the cosine of that
    row's cone angle to turn the oblique line integral into a transaxial one), over the turn of views
    whose source heights are centred on the slice, followed by fan-beam FBP.
    geom: HelicalConeGeometry with a whole number of views per turn; sino: [na][nt][ns].
    """
    g = geom
    turns = g.orbit_deg / 360.0
    na_turn = int(round(g.na / turns))
    if turns < 1.0 or abs(na_turn * turns - g.na) > 1e-9 * g.na:
        raise ValueError("need at least one turn and a whole number of views per turn")
    zk = (k - (g.nz - 1) / 2.0 + g.offset_z) * g.dz
    betas = g.betas()
    zsrc = np.array([g.source_z(b) for b in betas])
    vc = int(np.argmin(np.abs(zsrc - zk)))
    v0 = min(max(vc - na_turn // 2, 0), g.na - na_turn)
    p = np.empty((na_turn, g.ns), dtype=np.float64)
    c_row = (g.nt - 1) / 2.0 - g.offset_t  # row coordinate of detector height 0
    for i in range(na_turn):
        v = v0 + i
        h = (zk - zsrc[v]) * g.dsd / g.dso  # the slice's height at the isocentre, on the detector
        tc = min(max(h / g.dt + c_row, 0.0), g.nt - 1.0)
        t0 = min(int(math.floor(tc)), max(g.nt - 2, 0))
        f = tc - t0
        row = np.asarray(sino[v, t0], dtype=np.float64)
        if g.nt > 1:
            row = (1.0 - f) * row + f * np.asarray(sino[v, t0 + 1], dtype=np.float64)
        hc = (tc - c_row) * g.dt
        p[i] = row * (g.dsd / math.hypot(g.dsd, hc))
    return v0, p


def fbp_helical_ssrb(geom, sino: np.ndarray, window: str = "hann") -> np.ndarray:
    """Start image [nz][ny][nx] of a helical scan: per slice, single-slice rebinning (ssrb_sinogram)
    and the fan-beam FBP of that turn (fbp_fan_arc)."""
    g = geom
    turns = g.orbit_deg / 360.0
    na_turn = int(round(g.na / turns))
    out = np.empty((g.nz, g.ny, g.nx), dtype=np.float64)
    for k in range(g.nz):
        v0, p = ssrb_sinogram(g, sino, k)
        g2 = g.transaxial().with_(na=na_turn, orbit_deg=360.0,
                                  orbit_start_deg=g.orbit_start_deg + v0 * g.orbit_deg / g.na)
        out[k] = fbp_fan_arc(g2, p, window)
    return out
