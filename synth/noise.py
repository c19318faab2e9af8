"""Transmission noise model: Poisson photon counts plus Gaussian electronic noise.

counts = Poisson(I0 exp(-l)) + N(0, sigma_e^2), clamped to >= 1;
y = -log(counts / I0) (the noisy sinogram) and w = counts (statistical weights).
"""

from __future__ import annotations

import dataclasses

import numpy as np

from .configs import ScanConfig
from .phantom import anthropomorphic_ellipses, fan_arc_line_integrals, random_ellipses_cfg1
from .rng import philox


@dataclasses.dataclass
class SinoData:
    y: np.ndarray  # [na][ns] float64, -log(counts/I0)
    w: np.ndarray  # [na][ns] float64, counts (>= 1)
    line_integrals: np.ndarray  # noiseless bin-averaged line integrals
    ellipses: list


def transmission_data(line_integrals: np.ndarray, i0: float, sigma_e: float, seed: int) -> tuple[np.ndarray, np.ndarray]:
    rng = philox(seed, stream=303)
    mean = i0 * np.exp(-line_integrals)
    counts = rng.poisson(mean).astype(np.float64) + rng.normal(0.0, sigma_e, size=mean.shape)
    counts = np.maximum(counts, 1.0)
    y = -np.log(counts / i0)
    return y, counts


def make_scan(cfg: ScanConfig, n_gauss: int = 8) -> SinoData:
    """Phantom -> analytic sinogram -> noisy (y, w) for a workload configuration."""
    if cfg.phantom == "random10":
        E = random_ellipses_cfg1(cfg.seed)
    elif cfg.phantom == "anthro":
        E = anthropomorphic_ellipses(cfg.seed)
    else:
        raise ValueError(cfg.phantom)
    li = fan_arc_line_integrals(E, cfg.geom, n_gauss=n_gauss)
    y, w = transmission_data(li, cfg.i0, cfg.sigma_e, cfg.seed)
    return SinoData(y=y, w=w, line_integrals=li, ellipses=E)
