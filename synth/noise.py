"""Transmission noise model: Poisson photon counts plus Gaussian electronic noise.

counts = Poisson(I0 exp(-l)) + N(0, sigma_e^2), clamped to >= 1;
y = -log(counts / I0) (the noisy sinogram) and w = counts (statistical weights).
"""

from __future__ import annotations

import dataclasses

import numpy as np

from .configs import HelicalConeGeometry, ScanConfig
from .phantom import anthropomorphic_ellipses, fan_arc_line_integrals, random_ellipses_cfg1
from .phantom3d import anthropomorphic_solids, helical_line_integrals, random_solids
from .rng import philox


@dataclasses.dataclass
class SinoData:
    y: np.ndarray  # [na][ns] (helical: [na][nt][ns]) float64, -log(counts/I0)
    w: np.ndarray  # same shape, counts (>= 1)
    line_integrals: np.ndarray  # noiseless bin-averaged line integrals
    ellipses: list


def transmission_data(line_integrals: np.ndarray, i0: float, sigma_e: float, seed: int) -> tuple[np.ndarray, np.ndarray]:
    rng = philox(seed, stream=303)
    mean = i0 * np.exp(-line_integrals)
    counts = rng.poisson(mean).astype(np.float64) + rng.normal(0.0, sigma_e, size=mean.shape)
    counts = np.maximum(counts, 1.0)
    y = -np.log(counts / i0)
    return y, counts


def phantom_of(cfg: ScanConfig) -> list:
    """The seeded phantom (ellipses in 2-D, solids in 3-D) of a workload configuration."""
    g = cfg.geom
    if cfg.phantom == "random10":
        return random_ellipses_cfg1(cfg.seed)
    if cfg.phantom == "anthro":
        return anthropomorphic_ellipses(cfg.seed)
    if cfg.phantom == "random3d":
        return random_solids(cfg.seed, 0.45 * min(g.nx * g.dx, g.ny * g.dy), 0.45 * g.nz * g.dz)
    if cfg.phantom == "anthro3d":
        return anthropomorphic_solids(cfg.seed, 0.5 * g.nz * g.dz - 1.0)
    raise ValueError(cfg.phantom)


def make_scan(cfg: ScanConfig, n_gauss: int = 8, n_sub: int = 2) -> SinoData:
    """Phantom -> analytic sinogram -> noisy (y, w) for a workload configuration.

    2-D scans average ``n_gauss`` Gauss-Legendre rays per bin; helical scans
    ``n_sub x n_sub`` rays per detector cell.
    """
    E = phantom_of(cfg)
    if isinstance(cfg.geom, HelicalConeGeometry):
        li = helical_line_integrals(E, cfg.geom, n_sub=n_sub)
    else:
        li = fan_arc_line_integrals(E, cfg.geom, n_gauss=n_gauss)
    y, w = transmission_data(li, cfg.i0, cfg.sigma_e, cfg.seed)
    return SinoData(y=y, w=w, line_integrals=li, ellipses=E)
