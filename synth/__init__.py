"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package only *generates* inputs: scan geometries, ellipse/ellipsoid
phantoms, their analytic (closed-form) line integrals, and the transmission
noise model.  It holds none of the reconstruction method's arithmetic (no
projector matrix, regularizer or solver step), so that the FP64 oracle and
the GPU path can both consume the same inputs without sharing code.

Random numbers come from numpy's Philox counter-based generator (Salmon et
al., "Parallel random numbers: as easy as 1, 2, 3", SC 2011), keyed by the
caller's seed.
"""

from .configs import (FanArcGeometry, HelicalConeGeometry, ScanConfig, fan2d_128, fan2d_512, helix3d_64,
                      helix3d_512, config_by_name, warmstart_geometry)
from . import warmstart
from .phantom import (
    Ellipse,
    random_ellipses_cfg1,
    anthropomorphic_ellipses,
    rasterize_ellipses,
    fan_arc_line_integrals,
    fan_arc_line_integrals_sampled,
)
from .phantom3d import (
    Ellipsoid,
    EllipticCylinder,
    random_solids,
    anthropomorphic_solids,
    rasterize_solids,
    helical_line_integrals,
    helical_line_integrals_sampled,
)
from .noise import transmission_data, make_scan, phantom_of, SinoData
from .rng import philox

__all__ = [
    "FanArcGeometry",
    "HelicalConeGeometry",
    "ScanConfig",
    "helix3d_64",
    "helix3d_512",
    "Ellipsoid",
    "EllipticCylinder",
    "random_solids",
    "anthropomorphic_solids",
    "rasterize_solids",
    "helical_line_integrals",
    "helical_line_integrals_sampled",
    "phantom_of",
    "warmstart_geometry",
    "warmstart",
    "fan2d_128",
    "fan2d_512",
    "config_by_name",
    "Ellipse",
    "random_ellipses_cfg1",
    "anthropomorphic_ellipses",
    "rasterize_ellipses",
    "fan_arc_line_integrals",
    "fan_arc_line_integrals_sampled",
    "transmission_data",
    "SinoData",
    "make_scan",
    "philox",
]
