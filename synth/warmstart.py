"""Seeded problems of the learned-warm-start workload (inputs only).

Each problem is a chest-like ellipse phantom (its own seed: jittered organ
sizes, lesions) scanned with the warm-start geometry at an incident flux I0
drawn log-uniformly from [2e4, 2e5], with the transmission noise model of
``synth.noise`` (y = -log(counts / I0), w = counts).
"""

from __future__ import annotations

import math

import numpy as np

from .configs import FanArcGeometry
from .noise import transmission_data
from .phantom import anthropomorphic_ellipses, fan_arc_line_integrals
from .rng import philox


def problem(seed: int, g: FanArcGeometry, n_gauss: int = 2):
    """(y, w) float32 [na][ns] and the I0 of problem ``seed``."""
    rng = philox(seed, stream=606)
    i0 = float(math.exp(rng.uniform(math.log(2e4), math.log(2e5))))
    field = min(g.nx * g.dx, g.ny * g.dy) / 501.76  # the phantom fills a ~500 mm field at scale 1
    E = anthropomorphic_ellipses(10_000 + seed, scale=field * float(rng.uniform(0.85, 1.05)))
    li = fan_arc_line_integrals(E, g, n_gauss=n_gauss)
    y, w = transmission_data(li, i0, 5.0, 20_000 + seed)
    return y.astype(np.float32), w.astype(np.float32), i0


def _one(args):
    seed, g, n_gauss = args
    y, w, _ = problem(seed, g, n_gauss)
    return y, w


def problems(seeds, g: FanArcGeometry, n_gauss: int = 2, processes: int = 1):
    """Stacked (y, w) [len(seeds)][na][ns] for the given seeds (a spawn pool when processes > 1)."""
    jobs = [(int(s), g, n_gauss) for s in seeds]
    if processes > 1:
        import multiprocessing as mp

        with mp.get_context("spawn").Pool(processes) as pool:
            out = pool.map(_one, jobs, chunksize=max(1, len(jobs) // (4 * processes)))
    else:
        out = [_one(j) for j in jobs]
    return np.stack([o[0] for o in out]), np.stack([o[1] for o in out])
