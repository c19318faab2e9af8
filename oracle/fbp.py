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
