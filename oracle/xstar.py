"""Converged PWLS solution x* of a workload, computed by the oracle solver alone.

ORACLE -- test infrastructure only.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline / reference legs may import this module.

x* is the minimizer of the PWLS cost of Sec. III (Eq. (ct_problem)); with
beta > 0 and the strictly convex hyperbola potential it is unique.  It is
reached by relaxed OS-LALM (Algorithm 1 of Sec. III-A): ``os_iters`` outer
iterations with M ordered subsets from the FBP image (fast early progress),
then ``m1_iters`` iterations with one subset (ordered subsets stall in a limit
cycle; with M = 1 the method converges, Sec. III), restarted with rho = 1.
The result is accepted by the RMS of the projected-gradient fixed-point
residual (``solver.kkt_residual``) inside the field of view.

Running this module as a script writes ``oracle/data/xstar_<workload>_seed<k>.npy``
(float32, [ny][nx]) and a ``.json`` record of the recipe beside it.
"""

from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

from . import solver
from .fbp import fbp_fan_arc
from .projector import FanProjector, num_threads

HERE = os.path.dirname(os.path.abspath(__file__))
DATA = os.path.join(HERE, "data")


def path_for(name: str, seed: int) -> str:
    return os.path.join(DATA, f"xstar_{name}_seed{seed}.npy")


def compute(cfg, y, w, os_iters=20, M=20, m1_iters=400, alpha=1.999, log=None):
    """x* of the problem (y, w as float32 data of cfg's geometry); returns (x*, KKT RMS in HU)."""
    g = cfg.geom
    prob = solver.PWLSProblem(FanProjector(g), np.asarray(y, np.float64), np.asarray(w, np.float64),
                              cfg.beta_per_mm, cfg.delta, cfg.potential)
    DL = prob.D_L()
    x = fbp_fan_arc(g, prob.y, "hann")
    t0 = time.perf_counter()

    def cb(k, xk):
        if log:
            log(f"outer iteration {k}: {time.perf_counter() - t0:.0f} s")

    x = solver.relaxed_os_lalm(prob, x, M, alpha, os_iters, D_L=DL, callback=cb)
    x = solver.relaxed_os_lalm(prob, x, 1, alpha, m1_iters, D_L=DL, callback=cb)
    mask = solver.fov_mask(g)
    res = solver.kkt_residual(prob, x, D=DL + prob.D_R(x))
    kkt = float(np.sqrt(np.mean(res[mask] ** 2))) * cfg.hu_per_unit
    return x, kkt


def main(argv):
    sys.path.insert(0, os.path.dirname(HERE))
    import synth

    name = argv[1] if len(argv) > 1 else "fan2d_512"
    seed = int(argv[2]) if len(argv) > 2 else 0
    os_iters = int(argv[3]) if len(argv) > 3 else 20
    m1_iters = int(argv[4]) if len(argv) > 4 else 400
    cfg = synth.config_by_name(name, seed)
    d = synth.make_scan(cfg)
    M = max(1, cfg.M // 2)
    t0 = time.perf_counter()
    x, kkt = compute(cfg, d.y.astype(np.float32), d.w.astype(np.float32), os_iters=os_iters, M=M,
                     m1_iters=m1_iters, log=lambda s: print(s, flush=True))
    os.makedirs(DATA, exist_ok=True)
    p = path_for(name, seed)
    np.save(p, x.astype(np.float32))
    rec = {"workload": name, "seed": seed, "recipe": f"FBP, {os_iters} its of M={M}, {m1_iters} its of M=1 "
           "(relaxed OS-LALM, alpha 1.999, continuation)", "kkt_rms_hu": kkt,
           "seconds": round(time.perf_counter() - t0, 1), "threads": num_threads()}
    with open(p[:-4] + ".json", "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec), flush=True)


if __name__ == "__main__":
    main(sys.argv)
