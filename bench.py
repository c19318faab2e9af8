#!/usr/bin/env python
"""Benchmark: time for relaxed OS-LALM to reach RMSD <= 1 HU vs x* on one GB300.

Workload (default): 2-D fan beam at clinical scale -- 512x512 image, 0.98 mm
pixels, 888 bins x 1.0239 mm, 984 views, source-iso 541 mm, source-detector
949 mm; seeded chest-like ellipse phantom (mu in [0, 0.025]/mm); Poisson
I0 = 1e5 plus Gaussian electronic noise (sigma 5), W = counts; hyperbola
potential delta = 10 HU over 8 neighbours; relaxed OS-LALM with alpha =
1.999 and 30 iterations.  The workload names M = 41 subsets; relaxed OS-LALM
uses half the subsets of its unrelaxed counterpart (Sec. III-A), so the
timed solve uses M = 20, and the M = 41 traces (alpha 1.999 and 1) are
reported beside it.  x* comes from 2000 iterations of the same
(oracle-checked) solver with M = 1.

The scan's system matrix is built once per geometry (ct_geom_precompute,
timed separately) and stays resident in HBM.  One step = one whole solve
(D_L, initialisation, outer iterations) on device-resident inputs; `value` is
the mean device time from the solve's start to the end of the first
iteration whose RMSD to x* is <= 1 HU.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

def max_over_ranks(value, dist=None, device="cpu"):
    """The slowest rank's value, the same on every rank (None, a run that did not reach the tolerance,
    counts as infinitely slow and stays None).  dist: torch.distributed or None for one process; device:
    where the reduction tensor lives ("cuda" under NCCL, "cpu" under gloo)."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value if value is not None else float("inf")], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    v = float(t.item())
    return v if math.isfinite(v) else None


METRIC = "time to RMSD<=1 HU vs x* (s)"
UNIT = "s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fan2d_512")
    ap.add_argument("--alpha", type=float, default=None)
    ap.add_argument("--M", type=int, default=None)
    ap.add_argument("--n-iter", type=int, default=None)
    ap.add_argument("--xstar-iters", type=int, default=2000)
    ap.add_argument("--xstar-iters-batch", type=int, default=500,
                    help="batch workload x*: M = 1 iterations after 20 ordered-subsets iterations from the FBP")
    ap.add_argument("--tol-hu", type=float, default=1.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the warm-start and batched entries of the default line")
    ap.add_argument("--no-matrix", action="store_true", help="footprints on the fly instead of the resident matrix")
    ap.add_argument("--x0", default="fbp", choices=["fbp", "zeros"],
                    help="initial image: Hann-windowed FBP of the data (timed inside the solve) or zeros")
    ap.add_argument("--kernels-only", action="store_true",
                    help="only time one subset forward and back projection (profiling mode)")
    ap.add_argument("--views", type=int, default=None,
                    help="override the number of views over 360 deg (profiling smaller cases)")
    ap.add_argument("--study", action="store_true",
                    help="relaxed (alpha=1.999, M) vs unrelaxed (alpha=1, 2M) subsets, Algorithm 2 and fixed rho")
    ap.add_argument("--ws-train", type=int, default=2000, help="warm-start workload: training problems")
    ap.add_argument("--ws-eval", type=int, default=200, help="warm-start workload: held-out problems")
    ap.add_argument("--ws-epochs", type=int, default=12)
    ap.add_argument("--ws-batch", type=int, default=16)
    ap.add_argument("--ws-xstar-iters", type=int, default=400, help="M = 1 iterations of the held-out x*")
    ap.add_argument("--axial", default="rect", choices=["rect", "trap"],
                    help="helical workloads: axial footprint, rectangle (SF-TR) or trapezoid (SF-TT)")
    ap.add_argument("--xstar-iters-helix", type=int, default=600,
                    help="M = 1 iterations (after 40 iterations with a quarter of the subsets) for the helical x*")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [s.strip() for s in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_problem(args, rank: int):
    cfg = synth.config_by_name(args.workload, seed=rank)
    if args.views is not None:
        import dataclasses

        cfg = dataclasses.replace(cfg, geom=cfg.geom.with_(na=args.views))
    alpha = args.alpha if args.alpha is not None else cfg.alpha
    # relaxed OS-LALM: half the subsets of the unrelaxed method (Sec. III-A)
    M = args.M if args.M is not None else (max(1, cfg.M // 2) if alpha > 1.0 else cfg.M)
    n_iter = args.n_iter if args.n_iter is not None else cfg.n_iter
    data = synth.make_scan(cfg)
    return cfg, alpha, M, n_iter, data


def oracle_xstar(cfg):
    """The oracle's own x* of a workload (oracle/xstar.py; stored with its recipe), or None."""
    from oracle import xstar as oxstar

    p = oxstar.path_for(cfg.name, cfg.seed)
    if not os.path.exists(p):
        return None, None
    rec = {}
    try:
        rec = json.load(open(p[:-4] + ".json"))
    except (OSError, ValueError):
        pass
    return np.load(p).astype(np.float64), rec


def oracle_solve_to_tol(cfg, data, alpha, M, xstar, tol_hu, x0="fbp", max_iter=60, stop_after_sub=None):
    """One whole FP64 oracle solve, timed: FBP start (or zeros), D_L, the initial gradient, then outer
    iterations of Algorithm 1 until the RMSD to ``xstar`` over the FOV is <= tol_hu (checked after each
    outer iteration, as the GPU solver does).  stop_after_sub: end after that many subiterations (a
    bounded warm-up).  Returns the wall times and the iteration count."""
    from oracle import solver as osolver
    from oracle.projector import FanProjector, num_threads

    g = cfg.geom

    class Stop(Exception):
        pass

    t_start = time.perf_counter()
    prob = osolver.PWLSProblem(FanProjector(g), data.y.astype(np.float32).astype(np.float64),
                               data.w.astype(np.float32).astype(np.float64), cfg.beta_per_mm, cfg.delta,
                               cfg.potential)
    xinit = np.zeros((g.ny, g.nx))
    if x0 == "fbp":
        from oracle.fbp import fbp_fan_arc

        xinit = fbp_fan_arc(g, prob.y, "hann")
    t_fbp = time.perf_counter() - t_start
    DL = prob.D_L()
    t_dl = time.perf_counter() - t_start - t_fbp
    mask = osolver.fov_mask(g)
    out = {"iters_to_tol": None, "rmsd_trace_hu": []}

    def cb(k, x):
        r = osolver.rmsd_hu(x, xstar, mask, cfg.hu_per_unit)
        out["rmsd_trace_hu"].append(round(r, 4))
        if r <= tol_hu:
            out["iters_to_tol"] = k
            raise Stop()

    def sub_cb(t, x):
        if stop_after_sub is not None and t >= stop_after_sub:
            raise Stop()

    try:
        osolver.relaxed_os_lalm(prob, xinit, M, alpha, max_iter, D_L=DL, callback=cb, sub_callback=sub_cb)
    except Stop:
        pass
    out.update({"seconds": time.perf_counter() - t_start, "fbp_s": t_fbp, "dl_s": t_dl, "cores": num_threads()})
    return out


BATCH_SIZES = (256, 384, 512)
BATCH_BINS = (444, 888)
BATCH_VIEWS = (360, 492, 984)
BATCH_M = (10, 20, 41)


def _batch_slice(i):
    """Slice i of the 64-slice batch: (geometry, y, w, M); a 500 mm field of view in every case."""
    rng = synth.philox(i, stream=404)
    N = int(rng.choice(BATCH_SIZES))
    ns = int(rng.choice(BATCH_BINS))
    na = int(rng.choice(BATCH_VIEWS))
    M = int(rng.choice(BATCH_M))
    g = synth.FanArcGeometry(nx=N, ny=N, dx=0.98 * 512 / N, dy=0.98 * 512 / N, ns=ns, ds=1.0239 * 888 / ns, na=na,
                             dso=541.0, dsd=949.0)
    E = synth.anthropomorphic_ellipses(1000 + i)
    li = synth.fan_arc_line_integrals(E, g, n_gauss=2)
    y, w = synth.transmission_data(li, 1e5, 5.0, 1000 + i)
    return g, y.astype(np.float32), w.astype(np.float32), M


def batch_result(args, n_iter=100):
    """64 slices of mixed size, relaxed OS-LALM from the FBP start: the time for every slice to reach RMSD <=
    tol of its x*, solved in one batched call (persistent launch for the small slices) against a loop of
    single-slice solves that each stop at the tolerance.  Both forms are timed at the same accuracy: the
    batched call stops each slice at its first iteration at tol (the launch ends when all have) and its time
    is the device time from the call's start to the last slice's iteration at tol; the loop's is the sum of
    the single solves' times to tol.  Returns the result as a dict."""
    import multiprocessing as mp

    n = 64
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        slices = pool.map(_batch_slice, range(n))
    import torch

    from paper_1512_04564_gb300 import ct

    cfg = synth.fan2d_512()
    beta, delta, hu = cfg.beta_per_mm, cfg.delta, cfg.hu_per_unit
    geoms, tuned, mat_bytes = {}, {}, 0
    t0 = time.perf_counter()
    for g, _, _, _ in slices:
        key = (g.nx, g.ns, g.na)
        if key not in geoms:
            G = ct.Geometry.from_fan(g)
            mat_bytes += ct.ct_geom_precompute(G)
            tuned[str(key)] = ct.ct_geom_autotune(G)
            geoms[key] = G
    t_geo = time.perf_counter() - t0
    G_l = [geoms[(g.nx, g.ns, g.na)] for g, _, _, _ in slices]
    ys = [torch.from_numpy(y).cuda() for _, y, _, _ in slices]
    ws = [torch.from_numpy(w).cuda() for _, _, w, _ in slices]
    # relaxed OS-LALM: half the named subsets (Sec. III-A), but at most 10, of at least 40 views each: with
    # fewer views per subset, or 20 subsets of 49 views on the 256 x 256 slices, the iterates diverge (the
    # FP64 oracle's as well)
    Ms = [max(1, min(M // 2, g.na // 40, 10)) for g, _, _, M in slices]
    common = dict(alpha=1.999, beta=beta, delta=delta)
    # x* per slice: 20 ordered-subsets iterations from the FBP, then M = 1 iterations; the change over the
    # last 100 of those measures how far x* still is from converged
    xst = [torch.zeros(g.ny, g.nx, device="cuda") for g, _, _, _ in slices]
    t0 = time.perf_counter()
    ct.ct_relaxed_oslalm_solve_batched(G_l, ys, ws, xst, [dict(M=Ms[i], n_iter=20, init_fbp=True, **common)
                                                          for i in range(n)])
    ct.ct_relaxed_oslalm_solve_batched(G_l, ys, ws, xst,
                                       [dict(M=1, n_iter=max(1, args.xstar_iters_batch - 100), **common)] * n)
    x_prev = [x.clone() for x in xst]
    ct.ct_relaxed_oslalm_solve_batched(G_l, ys, ws, xst, [dict(M=1, n_iter=100, **common)] * n)
    t_xstar = time.perf_counter() - t0
    xstar_last100 = [float(((a - b) ** 2).mean().sqrt()) * hu for a, b in zip(xst, x_prev)]
    params = [dict(M=Ms[i], n_iter=n_iter, x_ref=xst[i], hu_per_unit=hu, init_fbp=True, stop_rmsd_hu=args.tol_hu,
                   **common) for i in range(n)]
    steps = max(1, min(args.steps, 3))
    for _ in range(max(1, min(args.warmup, 2))):
        xs = [torch.zeros_like(x) for x in xst]
        ct.ct_relaxed_oslalm_solve_batched(G_l, ys, ws, xs, params)
    b_tol, b_all, reps = [], [], None
    for _ in range(steps):
        xs = [torch.zeros_like(x) for x in xst]
        torch.cuda.synchronize()
        reps = ct.ct_relaxed_oslalm_solve_batched(G_l, ys, ws, xs, params)
        ttol = [r["seconds_to_tol"] for r in reps]
        b_tol.append(max(ttol) if all(t > 0 for t in ttol) else None)
        b_all.append(reps[0]["seconds"])
    # loop of single-slice solves (same parameters, CUDA-graph solver), each stopping at the tolerance
    l_tol, l_small = [], []
    solo = [i for i, (g, _, _, _) in enumerate(slices) if g.nx * g.ny >= 384 * 384]
    for _ in range(steps):
        tot, small, ok = 0.0, 0.0, True
        for i in range(n):
            x = torch.zeros_like(xst[i])
            r = ct.ct_relaxed_oslalm_solve(G_l[i], ys[i], ws[i], x, **params[i])
            ok = ok and r["seconds_to_tol"] > 0
            ti = r["seconds_to_tol"] if r["seconds_to_tol"] > 0 else r["seconds"]
            tot += ti
            if i not in solo:
                small += ti
        l_tol.append(tot if ok else None)
        l_small.append(small)
    # the batched call's path: slices of several geometries all run the single-slice solver on concurrent
    # lanes; one geometry's large slices alone, then one persistent launch for the rest
    several = len({id(G) for G in G_l}) > 1
    solo_end = max((reps[i]["seconds_to_tol"] for i in solo), default=0.0)
    shared_end = max((reps[i]["seconds_to_tol"] for i in range(n) if i not in solo), default=0.0)
    reached = sum(1 for r in reps if r["seconds_to_tol"] > 0)
    short = [{"slice": i, "image": slices[i][0].nx, "bins": slices[i][0].ns, "views": slices[i][0].na, "M": Ms[i],
              "min_rmsd_hu": round(min(r["rmsd_trace_hu"]), 3), "last_rmsd_hu": round(r["rmsd_trace_hu"][-1], 3),
              "xstar_change_last100_hu": round(xstar_last100[i], 4)}
             for i, r in enumerate(reps) if r["seconds_to_tol"] <= 0]
    iters = []
    for r in reps:
        tr = r["rmsd_trace_hu"]
        iters.append(next((i + 1 for i, v in enumerate(tr) if v <= args.tol_hu), None))
    bt = statistics.mean(b_tol) if all(v is not None for v in b_tol) else None
    lt = statistics.mean(l_tol) if all(v is not None for v in l_tol) else None
    out = {
        "workload": "batch64", "sizes": BATCH_SIZES, "bins": BATCH_BINS, "views": BATCH_VIEWS,
        "M_named": BATCH_M, "M_rule": "min(M//2, views//40, 10)", "alpha": 1.999, "n_iter_max": n_iter,
        "x0": "fbp", "xstar": f"20 its M from FBP + {args.xstar_iters_batch} its M=1",
        "xstar_change_last100_hu": {"median": statistics.median(xstar_last100), "max": max(xstar_last100)},
        "slices": n, "slices_reaching_tol": reached, "slices_short_of_tol": short,
        "iters_to_tol": {"median": statistics.median([i for i in iters if i]) if any(iters) else None,
                         "max": max([i for i in iters if i], default=None)},
        "batched_seconds_to_all_at_tol": bt, "loop_seconds_to_all_at_tol": lt,
        "batched_over_loop": (bt / lt) if bt and lt else None,
        "batched_seconds_full_call": statistics.mean(b_all),
        "parts": {"path": ("every slice on concurrent lanes (several geometries)" if several else
                           "large slices alone, then one persistent launch"),
                  "large_slices": len(solo),
                  "batched_large_alone_s": None if several else solo_end,
                  "batched_persistent_launch_s": None if several else shared_end - solo_end,
                  "loop_small_slices_s": statistics.mean(l_small),
                  "loop_large_slices_s": (statistics.mean(l_tol) - statistics.mean(l_small)) if lt else None},
        "geometries": len(geoms), "resident_matrix_bytes": mat_bytes, "geometry_setup_s": round(t_geo, 3),
        "autotuned": tuned, "xstar_seconds": round(t_xstar, 2), "steps": steps,
    }
    del geoms, G_l
    return out


def run_batch(args):
    """The batched workload as its own bench line."""
    import torch

    torch.cuda.set_device(0)
    clocks = ClockSampler(0)
    clocks.start()
    res = batch_result(args)
    clock_info = clocks.stop()
    v = res["batched_seconds_to_all_at_tol"]
    line = {
        "metric": METRIC + ", 64 slices batched", "value": v, "unit": UNIT, "n_gpus": 1, "steps": res["steps"],
        "warmup": args.warmup, "ms_per_step": v * 1e3 if v else None, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": res,
        "clocks": clock_info,
    }
    print(json.dumps(line), flush=True)
    return 0


def _helix_views(job):
    """Analytic line integrals of views [v0, v1) of a helical workload (worker of a spawn pool)."""
    name, seed, v0, v1 = job
    cfg = synth.config_by_name(name, seed)
    S = synth.phantom_of(cfg)
    return synth.helical_line_integrals(S, cfg.geom, n_sub=1, views=np.arange(v0, v1))


def helix_alu_roofline(ct, G, g, M, x, peaks, clock_mhz):
    """Subset forward / back projection of a helical scan: device time (CUDA events on the launching
    stream) against the FP32 FMA peak.  Algorithmic FLOPs = FLOP_PER_AIJ_3D per nonzero a_ij of the
    subset's rows, counted exactly on the host for a sample of the subset's views and scaled."""
    import torch

    views = list(range(M - 1, g.na, M))
    nv = len(views)
    out = torch.empty(nv, g.nt, g.ns, device="cuda")
    xb = torch.empty_like(x)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=10):
        for _ in range(3):
            fn()
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps * 1e-3

    fp_s = timed(lambda: ct.ct_forward(G, x, out, views=views))
    bp_s = timed(lambda: ct.ct_back(G, out, xb, views=views))
    sample = views[:: max(1, nv // 8)]
    nnz = sum(helix_nnz_view(g, v) for v in sample) * nv / len(sample)
    flops = FLOP_PER_AIJ_3D * nnz
    peak, peak_src = fp32_peak_tflops(clock_mhz)
    k = {"fp": {"kernel": "fp_helix_kernel", "ms": fp_s * 1e3, "tflops": flops / fp_s / 1e12},
         "bp": {"kernel": "bp_helix_kernel", "ms": bp_s * 1e3, "tflops": flops / bp_s / 1e12}}
    dom = "bp" if bp_s >= fp_s else "fp"
    return {"bound": "alu", "kernel": k[dom]["kernel"] + f" ({nv} views)", "achieved": k[dom]["tflops"],
            "peak": peak, "unit": "TFLOP/s", "frac": k[dom]["tflops"] / peak, "traffic": None,
            "peak_source": peak_src + " (derived from unit counts and the sampled clock)",
            "nnz_per_launch": nnz, "flop_per_aij": FLOP_PER_AIJ_3D, "views_per_launch": nv, "kernels": k}


def helix_nnz_view(g, v):
    """Number of nonzero a_ij in view v of a helical SF-TR matrix (transaxial cells x axial rows per voxel)."""
    b = g.betas()[v]
    cb, sb = math.cos(b), math.sin(b)
    xc = (np.arange(g.nx) - (g.nx - 1) / 2.0 + g.offset_x) * g.dx
    yc = (np.arange(g.ny) - (g.ny - 1) / 2.0 + g.offset_y) * g.dy
    X, Y = np.meshgrid(xc, yc)
    taus = []
    for sx in (-0.5, 0.5):
        for sy in (-0.5, 0.5):
            px, py = X + sx * g.dx + g.dso * cb, Y + sy * g.dy + g.dso * sb
            taus.append(np.arctan2(-px * sb + py * cb, px * cb + py * sb) * g.dsd / g.ds + (g.ns - 1) / 2.0 - g.offset_s)
    t0, t3 = np.minimum.reduce(taus), np.maximum.reduce(taus)
    s_lo = np.maximum(np.floor(t0 - 0.5) + 1, 0)
    s_hi = np.minimum(np.ceil(t3 + 0.5) - 1, g.ns - 1)
    cells = np.maximum(s_hi - s_lo + 1, 0)
    L = np.hypot(X + g.dso * cb, Y + g.dso * sb)
    zs = g.source_z(b)
    zc = (np.arange(g.nz) - (g.nz - 1) / 2.0 + g.offset_z) * g.dz
    c0 = (g.nt - 1) / 2.0 - g.offset_t
    u0 = ((zc[:, None, None] - 0.5 * g.dz - zs) * g.dsd / L[None]) / g.dt + c0
    u1 = ((zc[:, None, None] + 0.5 * g.dz - zs) * g.dsd / L[None]) / g.dt + c0
    rows = np.clip(np.ceil(u1 + 0.5) - 1, -1, g.nt - 1) - np.clip(np.floor(u0 - 0.5) + 1, 0, g.nt)
    rows = np.maximum(rows + 1, 0)
    return float((rows.sum(axis=0) * cells).sum())


def run_helix(args):
    """Helical cone-beam workload: relaxed OS-LALM time to RMSD <= 1 HU vs x*, with its ALU roofline."""
    import multiprocessing as mp

    cfg = synth.config_by_name(args.workload, 0)
    g = dataclasses.replace(cfg.geom, axial=args.axial)
    if args.kernels_only:
        import torch

        from paper_1512_04564_gb300 import ct

        torch.cuda.set_device(0)
        G = ct.Geometry.from_helix(g)
        S = synth.phantom_of(cfg)
        xk = torch.from_numpy(synth.rasterize_solids(S, g, oversample=1, oversample_z=1).astype(np.float32)).cuda()
        M = args.M or cfg.M
        roof = helix_alu_roofline(ct, G, g, M, xk, {}, None)
        print(json.dumps({"mode": "kernels-only", "workload": cfg.name, "axial": args.axial, "M": M, "roofline": roof}),
              flush=True)
        return 0
    t0 = time.perf_counter()
    step = max(1, g.na // 64)
    jobs = [(cfg.name, 0, v, min(v + step, g.na)) for v in range(0, g.na, step)]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        li = np.concatenate(pool.map(_helix_views, jobs), axis=0)
    y_np, w_np = synth.transmission_data(li, cfg.i0, cfg.sigma_e, cfg.seed)
    t_data = time.perf_counter() - t0
    import torch

    from paper_1512_04564_gb300 import ct

    torch.cuda.set_device(0)
    G = ct.Geometry.from_helix(g)
    y = torch.from_numpy(y_np.astype(np.float32)).cuda()
    w = torch.from_numpy(w_np.astype(np.float32)).cuda()
    beta, delta, hu = cfg.beta_per_mm, cfg.delta, cfg.hu_per_unit
    common = dict(beta=beta, delta=delta, potential=cfg.potential)
    shape = (g.nz, g.ny, g.nx)
    # x*: 40 iterations with a quarter of the named subsets (close to the minimizer in the low
    # frequencies, which M = 1 reaches slowly), then M = 1
    xstar = torch.zeros(shape, device="cuda")
    t0 = time.perf_counter()
    m_warm = max(1, cfg.M // 4)
    ct.ct_relaxed_oslalm_solve(G, y, w, xstar, M=m_warm, n_iter=40, alpha=1.999, **common)
    ct.ct_relaxed_oslalm_solve(G, y, w, xstar, M=1, n_iter=args.xstar_iters_helix, alpha=1.999, **common)
    torch.cuda.synchronize()
    t_xstar = time.perf_counter() - t0
    kkt = kkt_rms_hu(ct, G, g, y, w, xstar, beta, delta, cfg.potential, hu)
    # the workload names 20 iterations; the run continues to 60 so that the time to 1 HU is measured
    n_iter = args.n_iter or 3 * cfg.n_iter
    alpha = args.alpha or cfg.alpha
    # the named subset count, and fewer subsets (a lower ordered-subsets limit cycle)
    Ms = [args.M] if args.M else [cfg.M, cfg.M // 2, cfg.M // 4]

    fbp0 = args.x0 == "fbp"  # the rebinned slice-by-slice FBP (timed inside the solve), or zeros

    def solve(M):
        x = torch.zeros(shape, device="cuda")
        return ct.ct_relaxed_oslalm_solve(G, y, w, x, M=M, n_iter=n_iter, alpha=alpha, x_ref=xstar, hu_per_unit=hu,
                                          init_fbp=fbp0, **common)

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    runs = {}
    clocks = ClockSampler(0)
    clocks.start()
    for M in Ms:
        for _ in range(args.warmup):
            solve(M)
        reps = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            reps.append(solve(M))
        tr = reps[-1]["rmsd_trace_hu"]
        hit = next((i + 1 for i, r in enumerate(tr) if r <= args.tol_hu), None)
        ttol = [r["seconds_to_tol"] for r in reps]
        runs[M] = {"seconds_to_tol": statistics.mean(ttol) if all(t > 0 for t in ttol) else None,
                   "iters_to_tol": hit, "seconds_per_iter": statistics.mean(r["seconds"] for r in reps) / n_iter,
                   "rmsd_hu_at_named_iters": round(tr[min(cfg.n_iter, len(tr)) - 1], 3),
                   "rmsd_trace_hu": [round(r, 3) for r in tr]}
    clock_info = clocks.stop()
    best = min((m for m in runs if runs[m]["seconds_to_tol"]), key=lambda m: runs[m]["seconds_to_tol"], default=None)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    roof = helix_alu_roofline(ct, G, g, best or Ms[0], xstar, peaks, clock_info.get("sm_mhz"))
    line = {
        "metric": METRIC, "value": runs[best]["seconds_to_tol"] if best else None, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": cfg.name, "volume": list(shape), "voxel_mm": [g.dx, g.dy, g.dz],
                   "detector": [g.nt, g.ns], "views": g.na, "turns": g.orbit_deg / 360.0, "pitch": g.pitch,
                   "axial": args.axial,
                   "alpha": alpha, "n_iter": n_iter, "n_iter_named": cfg.n_iter, "M_named": cfg.M, "M_best": best,
                   "x0": "rebinned FBP" if fbp0 else "zeros",
                   "beta_water_units": cfg.beta, "xstar": f"40 its M={m_warm} + {args.xstar_iters_helix} its M=1",
                   "xstar_kkt_rms_hu": kkt, "l2": "flushed (256 MB write) between steps",
                   "data_generation_s": round(t_data, 2)},
        "runs_by_M": runs,
        "gpu_launches": n_iter * (3 * (best or Ms[0]) + 1) + 6,
        "roofline": roof,
        "clocks": clock_info,
        "xstar_seconds": t_xstar,
    }
    print(json.dumps(line), flush=True)
    return 0


def unet_flops(levels, base, H, W):
    """FLOPs of one U-Net forward per image (2 per multiply-add of the 3x3 layers and the 1x1 output)."""
    ch = [base << l for l in range(levels)]
    f = 0
    for l in range(levels):
        hw = (H >> l) * (W >> l)
        f += 2 * hw * 9 * ((1 if l == 0 else ch[l - 1]) * ch[l] + ch[l] * ch[l])
    for l in range(levels - 2, -1, -1):
        hw = (H >> l) * (W >> l)
        f += 2 * hw * 9 * ((ch[l + 1] + ch[l]) * ch[l] + ch[l] * ch[l])
    return f + 2 * H * W * base


def unet_roofline(ct, net, levels, base, H, W, B, peaks, clock_mhz):
    """Device time of one U-Net forward and one forward + backward at batch B (CUDA events), against the
    measured BF16 dense peak; the largest tensor-core layer alone is timed with the single-layer entry."""
    import torch

    x = torch.rand(B, H, W, device="cuda") * 0.02
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=10):
        for _ in range(3):
            fn()
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps * 1e-3

    gy = torch.randn(B, H, W, device="cuda")
    t_fwd = timed(lambda: ct.ct_unet_forward(net, x))

    def step():
        ct.ct_unet_forward(net, x)
        ct.ct_unet_backward(net, gy)

    t_step = timed(step)
    f_fwd = unet_flops(levels, base, H, W) * B
    f_step = 3 * f_fwd  # forward, input gradients, weight gradients
    # the largest layer: decoder level 0, conv a (upsampled 2 C0 + skip C0 -> C0) at full resolution
    c1, c2, co = 2 * base, base, base
    a1 = torch.randn(B, H // 2, W // 2, c1, device="cuda").to(torch.bfloat16)
    a2 = torch.randn(B, H, W, c2, device="cuda").to(torch.bfloat16)
    wl = (torch.randn(co, 9 * (c1 + c2), device="cuda") * 0.05).to(torch.bfloat16)
    bl = torch.zeros(co, device="cuda")
    out = torch.empty(B, H, W, co, dtype=torch.bfloat16, device="cuda")
    t_layer = timed(lambda: ct.ct_conv3x3_bf16(a1, c1, 1, a2, c2, wl, bl, out, B, H, W, co))
    f_layer = 2 * B * H * W * 9 * (c1 + c2) * co
    peak = peaks.get("bf16_tflops", 1900.0)
    k = {"unet_forward": {"ms": t_fwd * 1e3, "tflops": f_fwd / t_fwd / 1e12},
         "unet_train_step": {"ms": t_step * 1e3, "tflops": f_step / t_step / 1e12},
         "conv3x3_dec0a_forward": {"ms": t_layer * 1e3, "tflops": f_layer / t_layer / 1e12}}
    return {"bound": "tensor", "kernel": f"U-Net forward (batch {B}, {H}x{W}, tcgen05 BF16 convs)",
            "achieved": k["unet_forward"]["tflops"], "peak": peak, "unit": "TFLOP/s",
            "frac": k["unet_forward"]["tflops"] / peak, "traffic": None,
            "peak_source": "MEASURED_PEAKS.json bf16_tflops (measured, cuBLAS burst)" if peaks else "fallback 1900",
            "kernels": k}


def warmstart_result(args):
    """Learned warm start on the 256x256 workload: generate the problems (FBP -> x*), train the U-Net on the
    GPU, then relaxed OS-LALM to tol from the warm start vs the FBP start on the held-out problems.  Returns
    (result dict, the network, clocks during the evaluation)."""
    import torch

    n_train, n_eval = args.ws_train, args.ws_eval
    g = synth.warmstart_geometry(256)
    t0 = time.perf_counter()
    seeds = list(range(n_train)) + list(range(100_000, 100_000 + n_eval))
    y_np, w_np = synth.warmstart.problems(seeds, g, n_gauss=1, processes=min(16, os.cpu_count() or 1))
    t_data = time.perf_counter() - t0
    from paper_1512_04564_gb300 import ct, warmstart

    torch.cuda.set_device(0)
    G = ct.Geometry.from_fan(g)
    mat = ct.ct_geom_precompute(G)
    ys, ws = torch.from_numpy(y_np).cuda(), torch.from_numpy(w_np).cuda()
    del y_np, w_np
    cfg = synth.fan2d_512()
    beta, delta, hu = cfg.beta_per_mm, cfg.delta, cfg.hu_per_unit
    M = args.M or 10  # the workload names M = 20; relaxed OS-LALM uses half the subsets (Sec. III-A)
    t0 = time.perf_counter()
    xs_train = warmstart.solve_xstar(G, ys[:n_train], ws[:n_train], beta, delta, os_iters=15, m1_iters=40, M=M)
    xs_eval = warmstart.solve_xstar(G, ys[n_train:], ws[n_train:], beta, delta, os_iters=20,
                                    m1_iters=args.ws_xstar_iters, M=M)
    torch.cuda.synchronize()
    t_xstar = time.perf_counter() - t0
    kkt = [kkt_rms_hu(ct, G, g, ys[n_train + i], ws[n_train + i], xs_eval[i], beta, delta, cfg.potential, hu)
           for i in range(min(4, n_eval))]
    # the training targets' distance to a converged x* (on the first problems of the training set)
    ref = warmstart.solve_xstar(G, ys[:4], ws[:4], beta, delta, os_iters=20, m1_iters=args.ws_xstar_iters, M=M)
    X = (torch.arange(g.nx, device="cuda") - (g.nx - 1) / 2.0) * g.dx
    mask = (X[None, :] ** 2 + X[:, None] ** 2) <= g.fov_radius() ** 2
    tgt_err = [float(((xs_train[i] - ref[i])[mask].double().pow(2).mean().sqrt()) * hu) for i in range(4)]
    fbp = warmstart.fbp_images(G, ys)
    net = ct.UNet(levels=4, base_channels=32, height=256, width=256, max_batch=args.ws_batch, in_scale=1 / 0.02,
                  seed=0)
    t0 = time.perf_counter()
    hist = warmstart.train(net, G, fbp[:n_train], xs_train, ys[:n_train], ws[:n_train], epochs=args.ws_epochs,
                           batch=args.ws_batch, lr=2e-3, lr_min=5e-5, lam_dc=1e-4)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    clocks = ClockSampler(0)
    clocks.start()
    res = warmstart.evaluate(net, G, ys[n_train:], ws[n_train:], xs_eval, beta=beta, delta=delta, M=M, n_iter=40)
    clock_info = clocks.stop()
    res.pop("per_problem", None)
    out = {"warm_start_seconds": res["warm_seconds"]["mean"], "plain_start_seconds": res["plain_seconds"]["mean"],
           "workload": "warmstart256", "image": [256, 256], "bins": g.ns, "views": g.na,
           "train_problems": n_train, "eval_problems": n_eval, "I0": [2e4, 2e5], "M": M, "M_named": 20,
           "alpha": 1.999, "unet": {"levels": 4, "base_channels": 32, "params": net.num_params},
           "epochs": args.ws_epochs, "batch": args.ws_batch, "loss": "MSE (water units) + 1e-4 DC",
           "xstar_eval": f"20 its M={M} + {args.ws_xstar_iters} its M=1 from FBP",
           "xstar_train": f"15 its M={M} + 40 its M=1 from FBP",
           "xstar_kkt_rms_hu": kkt, "train_target_rmsd_to_xstar_hu": tgt_err, "resident_matrix_bytes": mat,
           "results": res, "train_loss_by_epoch": [round(h, 6) for h in hist],
           "timings_s": {"data_generation": round(t_data, 1), "xstar": round(t_xstar, 1),
                         "training": round(t_train, 1)}}
    return out, net, clock_info


def run_warmstart(args):
    """Learned warm start: 2000 generated 256x256 problems (FBP -> x*), training on the GPU, and iterations /
    seconds of relaxed OS-LALM to 1 HU from the warm start vs the FBP start on 200 held-out problems."""
    import torch

    from paper_1512_04564_gb300 import ct

    torch.cuda.set_device(0)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    if args.kernels_only:
        net = ct.UNet(levels=4, base_channels=32, height=256, width=256, max_batch=args.ws_batch, in_scale=50.0)
        roof = unet_roofline(ct, net, 4, 32, 256, 256, args.ws_batch, peaks, None)
        print(json.dumps({"mode": "kernels-only", "workload": "warmstart256", "roofline": roof}), flush=True)
        return 0
    res, net, clock_info = warmstart_result(args)
    roof = unet_roofline(ct, net, 4, 32, 256, 256, args.ws_batch, peaks, clock_info.get("sm_mhz"))
    line = {
        "metric": METRIC + ", learned warm start", "value": res["warm_start_seconds"], "unit": UNIT, "n_gpus": 1,
        "steps": res["eval_problems"], "warmup": 0, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 U-Net / f32 solver", "data": "synthetic", "config": res,
        "plain_start_seconds": res["plain_start_seconds"], "roofline": roof, "clocks": clock_info,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on the host cores.  Each timed step is one whole
    oracle solve to RMSD <= tol vs the oracle's own x* (FBP, D_L, initialisation, outer iterations with the
    RMSD checked after each); warm-up steps run the same solve for one subiteration."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cfg, alpha, M, n_iter, data = make_problem(args, 0)
    xstar, rec = oracle_xstar(cfg) if args.views is None else (None, None)
    if xstar is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no oracle x* stored for workload {cfg.name} "
                          "(oracle/xstar.py writes one)"}), flush=True)
        return 0
    for _ in range(args.warmup):
        oracle_solve_to_tol(cfg, data, alpha, M, xstar, args.tol_hu, x0=args.x0, stop_after_sub=1)
    runs = [oracle_solve_to_tol(cfg, data, alpha, M, xstar, args.tol_hu, x0=args.x0, max_iter=n_iter)
            for _ in range(args.steps)]
    reached = all(r["iters_to_tol"] is not None for r in runs)
    step_s = [r["seconds"] for r in runs]
    v = statistics.mean(step_s) if reached else None
    last = runs[-1]
    sample = (f"{args.steps} whole FP64 oracle solves (one per step): FBP {last['fbp_s']:.2f} s, D_L {last['dl_s']:.2f} s, "
              f"then {last['iters_to_tol']} outer iterations of M = {M} to RMSD <= {args.tol_hu} HU of the "
              f"oracle's x* ({rec.get('recipe', '?')}; KKT RMS {rec.get('kkt_rms_hu', float('nan')):.2e} HU)")
    cb = {"value": v, "unit": UNIT, "cores": last["cores"], "kind": "oracle", "sample": sample}
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(step_s) * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": cfg.name, "alpha": alpha, "M": M, "n_iter": n_iter, "x0": args.x0,
                   "iters_to_tol": [r["iters_to_tol"] for r in runs], "rmsd_trace_hu": last["rmsd_trace_hu"],
                   "warmup": "one subiteration of the same solve per warm-up step"},
        "cpu_baseline": cb,
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch(args)
    if args.workload.startswith("helix"):
        return run_helix(args)
    if args.workload == "warmstart256":
        return run_warmstart(args)

    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_1512_04564_gb300 import ct

    cfg, alpha, M, n_iter, data = make_problem(args, rank)
    g = cfg.geom
    G = ct.Geometry.from_fan(g)
    matrix_bytes, t_matrix = 0, 0.0
    if not args.no_matrix:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        matrix_bytes = ct.ct_geom_precompute(G)
        torch.cuda.synchronize()
        t_matrix = time.perf_counter() - t0
    y = torch.from_numpy(data.y.astype(np.float32)).cuda()
    w = torch.from_numpy(data.w.astype(np.float32)).cuda()
    beta, delta, hu = cfg.beta_per_mm, cfg.delta, cfg.hu_per_unit
    common = dict(beta=beta, delta=delta, potential=cfg.potential)
    if args.kernels_only:
        xk = torch.from_numpy(synth.rasterize_ellipses(data.ellipses, g.nx, g.ny, g.dx, g.dy,
                                                       oversample=1).astype(np.float32)).cuda()
        roof = kernel_roofline(ct, G, g, M, y, w, xk, matrix_bytes)
        if rank == 0:
            print(json.dumps({"mode": "kernels-only", "workload": cfg.name, "views": g.na, "M": M,
                              "matrix_bytes": matrix_bytes, "roofline": roof}), flush=True)
        return 0

    # x*: M = 1 relaxed LALM from zero, then its KKT residual
    xstar = torch.zeros(g.ny, g.nx, device="cuda")
    t0 = time.perf_counter()
    ct.ct_relaxed_oslalm_solve(G, y, w, xstar, M=1, n_iter=args.xstar_iters, alpha=1.999, **common)
    t_xstar = time.perf_counter() - t0
    kkt = kkt_rms_hu(ct, G, g, y, w, xstar, beta, delta, cfg.potential, hu)
    if args.study:
        return run_study(args, ct, G, g, y, w, xstar, common, hu, kkt, cfg)

    fbp0 = args.x0 == "fbp"

    def solve_once(stop=0.0):
        x = torch.zeros(g.ny, g.nx, device="cuda")
        rep = ct.ct_relaxed_oslalm_solve(G, y, w, x, M=M, n_iter=n_iter, alpha=alpha, x_ref=xstar, hu_per_unit=hu,
                                         stop_rmsd_hu=stop, init_fbp=fbp0, **common)
        return rep, x

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    for _ in range(args.warmup):
        rep, _ = solve_once()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    reps = []
    start_ev, end_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        barrier()
        start_ev.record()
        rep, _ = solve_once()
        end_ev.record()
        barrier()
        step_ms.append(start_ev.elapsed_time(end_ev))
        reps.append(rep)
    clock_info = clocks.stop()
    t_tol = [r["seconds_to_tol"] for r in reps]
    reached = all(t > 0 for t in t_tol)
    value = statistics.mean(t_tol) if reached else None
    iters_to_tol = None
    if reached:
        tr = reps[-1]["rmsd_trace_hu"]
        iters_to_tol = next(i + 1 for i, r in enumerate(tr) if r <= args.tol_hu)
    value = max_over_ranks(value, dist, "cuda")

    # e2e: host buffers in, result out, through the public API
    y_h = torch.from_numpy(data.y.astype(np.float32)).pin_memory()
    w_h = torch.from_numpy(data.w.astype(np.float32)).pin_memory()
    x_h = torch.empty(g.ny, g.nx, pin_memory=True)
    e2e_times = []
    for _ in range(max(2, args.steps)):
        flush.fill_(1.0)
        barrier()
        t0 = time.perf_counter()
        yd = y_h.to("cuda", non_blocking=True)
        wd = w_h.to("cuda", non_blocking=True)
        x = torch.zeros(g.ny, g.nx, device="cuda")
        ct.ct_relaxed_oslalm_solve(G, yd, wd, x, M=M, n_iter=n_iter, alpha=alpha, x_ref=xstar, hu_per_unit=hu,
                                   stop_rmsd_hu=args.tol_hu, init_fbp=fbp0, **common)
        x_h.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    e2e = {"value": max_over_ranks(statistics.mean(e2e_times), dist, "cuda"), "unit": UNIT,
           "h2d_bytes_per_step": 2 * y_h.numel() * 4,
           "d2h_bytes_per_step": x_h.numel() * 4}
    # e2e_cold: the same, with the geometry created (FP64 anchor tables) and its matrix built inside the
    # timed region, as for a scan geometry seen for the first time
    cold_times = []
    for _ in range(2):
        flush.fill_(1.0)
        barrier()
        t0 = time.perf_counter()
        G2 = ct.Geometry.from_fan(g)
        if matrix_bytes:
            ct.ct_geom_precompute(G2)
        yd = y_h.to("cuda", non_blocking=True)
        wd = w_h.to("cuda", non_blocking=True)
        x = torch.zeros(g.ny, g.nx, device="cuda")
        ct.ct_relaxed_oslalm_solve(G2, yd, wd, x, M=M, n_iter=n_iter, alpha=alpha, x_ref=xstar, hu_per_unit=hu,
                                   stop_rmsd_hu=args.tol_hu, init_fbp=fbp0, **common)
        x_h.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
        cold_times.append(time.perf_counter() - t0)
        G2.close()
    e2e_cold = {"value": max_over_ranks(statistics.mean(cold_times), dist, "cuda"), "unit": UNIT,
                "h2d_bytes_per_step": e2e["h2d_bytes_per_step"], "d2h_bytes_per_step": e2e["d2h_bytes_per_step"],
                "includes": "ct_geom_create + " + ("ct_geom_precompute + " if matrix_bytes else "") +
                            "the e2e solve through host buffers"}

    roof = kernel_roofline(ct, G, g, M, y, w, xstar, matrix_bytes, clock_info.get("sm_mhz"))
    # setup: D_L weights and back-projection, initial FP (+ packing [x | x^T] for the resident rows) and BP,
    # the FBP's filter and back-projection; then 3 launches per subiteration and the RMSD per iteration
    launches = 4 + (1 if matrix_bytes else 0) + (2 if fbp0 else 0) + n_iter * (3 * M + 1)
    # the workload's own subset count, for the record (untimed)
    m41 = {}
    if M != cfg.M:
        for a41 in (alpha, 1.0):
            x41 = torch.zeros(g.ny, g.nx, device="cuda")
            r41 = ct.ct_relaxed_oslalm_solve(G, y, w, x41, M=cfg.M, n_iter=n_iter, alpha=a41, x_ref=xstar,
                                             hu_per_unit=hu, init_fbp=fbp0, **common)
            tr = r41["rmsd_trace_hu"]
            hit = next((i + 1 for i, r in enumerate(tr) if r <= args.tol_hu), None)
            m41[f"alpha{a41:g}"] = {"iters_to_tol": hit, "min_rmsd_hu": round(min(tr), 3),
                                    "last_rmsd_hu": round(tr[-1], 3)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": max_over_ranks(statistics.mean(step_ms), dist, "cuda"), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": cfg.name, "image": [g.ny, g.nx], "views": g.na, "bins": g.ns, "M": M,
                   "alpha": alpha, "n_iter": n_iter, "M_named": cfg.M, "beta_water_units": cfg.beta,
                   "x0": args.x0, "xstar_iters": args.xstar_iters,
                   "system_matrix": {"resident": matrix_bytes > 0, "bytes": matrix_bytes, "build_s": round(t_matrix, 4)},
                   "M_named_runs": m41,
                   "xstar_kkt_rms_hu": kkt, "iters_to_tol": iters_to_tol, "l2": "flushed (256 MB write) between steps",
                   "parallelism": f"replicas{world}"},
        "gpu_launches": launches,
        "e2e": e2e,
        "e2e_cold": e2e_cold,
        "roofline": roof,
        "clocks": clock_info,
        "rmsd_trace_hu": [round(r, 4) for r in reps[-1]["rmsd_trace_hu"]],
        "xstar_seconds": t_xstar,
        "source_digest": _source_digest(),
    }
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        xs_o, rec = oracle_xstar(cfg) if args.views is None else (None, None)
        if xs_o is not None:
            # the oracle's own solve, once, to the same tolerance of its own x*
            r = oracle_solve_to_tol(cfg, data, alpha, M, xs_o, args.tol_hu, x0=args.x0, max_iter=n_iter)
            line["cpu_baseline"] = {
                "value": r["seconds"] if r["iters_to_tol"] else None, "unit": UNIT, "cores": r["cores"],
                "kind": "oracle",
                "sample": (f"one whole FP64 oracle solve: FBP {r['fbp_s']:.2f} s, D_L {r['dl_s']:.2f} s, then "
                           f"{r['iters_to_tol']} outer iterations of M = {M} to RMSD <= {args.tol_hu} HU of the "
                           f"oracle's x* ({rec.get('recipe', '?')})"),
                "rmsd_trace_hu": r["rmsd_trace_hu"]}
            # the two x* (GPU: M = 1 iterations; oracle: its stored recipe) of the same problem
            line["config"]["xstar_gpu_vs_oracle_rmsd_hu"] = float(
                np.sqrt(np.mean(((xstar.cpu().numpy() - xs_o)[fov_mask_np(g)]) ** 2)) * hu)
    if rank == 0 and world == 1 and not args.no_extras:
        # the learned warm start and the batched form, each timed to the same accuracy as the plain start
        try:
            ws_res, _, ws_clocks = warmstart_result(args)
            line["warm_start"] = {
                "value": ws_res["warm_start_seconds"], "plain_start_value": ws_res["plain_start_seconds"],
                "unit": UNIT, "metric": "mean device time to RMSD <= 1 HU of x* over the held-out problems, "
                                        "FBP and U-Net inference included",
                "config": {k: v for k, v in ws_res.items() if k not in ("results", "train_loss_by_epoch")},
                "results": ws_res["results"], "clocks": ws_clocks}
        except Exception as e:  # the headline line stands without it
            line["warm_start"] = {"error": repr(e)}
        try:
            line["batched"] = batch_result(args)
        except Exception as e:
            line["batched"] = {"error": repr(e)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_study(args, ct, G, g, y, w, xstar, common, hu, kkt, cfg):
    """The paper's comparisons on the synthetic workload, each as iterations and device seconds to 1 HU of x*
    from the FBP start: relaxed (alpha = 1.999) with M subsets against unrelaxed (alpha = 1) with M and 2M
    (Sec. IV: the relaxed method matches the unrelaxed one with about twice the subsets); the proposed
    relaxation (Algorithm 1) against the simple one (Algorithm 2), with continuation and with fixed rho = 0.05;
    and the supplement's majorizer study (maximum-curvature D_R; D_L scaled by 0.5 .. 4)."""
    import torch

    n_iter = args.n_iter or 40

    def run(M, alpha, algorithm="proposed", continuation=True, rho_fixed=0.0, curvature="huber", dl_scale=1.0):
        x = torch.zeros(g.ny, g.nx, device="cuda")
        r = ct.ct_relaxed_oslalm_solve(G, y, w, x, M=M, n_iter=n_iter, alpha=alpha, algorithm=algorithm,
                                       continuation=continuation, rho_fixed=rho_fixed, x_ref=xstar, hu_per_unit=hu,
                                       init_fbp=True, curvature=curvature, dl_scale=dl_scale, **common)
        tr = r["rmsd_trace_hu"]
        hit = next((i + 1 for i, v in enumerate(tr) if v <= args.tol_hu), None)
        return {"M": M, "alpha": alpha, "algorithm": algorithm,
                "rho": "continuation" if continuation else rho_fixed, "curvature": curvature, "dl_scale": dl_scale,
                "iters_to_1hu": hit,
                "seconds_to_1hu": r["seconds_to_tol"] if r["seconds_to_tol"] > 0 else None,
                "min_rmsd_hu": round(min(tr), 4), "rmsd_trace_hu": [round(v, 3) for v in tr]}

    for _ in range(2):  # warm-up of the graph path
        run(10, 1.999)
    pairs = [{"relaxed": run(M, 1.999), "unrelaxed": run(M, 1.0), "unrelaxed_2M": run(2 * M, 1.0)}
             for M in (5, 10, 20)]
    algs = [run(20, 1.999, "proposed"), run(20, 1.999, "simple"),
            run(20, 1.999, "proposed", continuation=False, rho_fixed=0.05),
            run(20, 1.999, "simple", continuation=False, rho_fixed=0.05)]
    majorizers = [run(20, 1.999, curvature="max")] + [run(20, 1.999, dl_scale=k) for k in (0.5, 0.75, 2.0, 4.0)]
    line = {"mode": "study", "workload": cfg.name, "x0": "fbp", "n_iter": n_iter, "xstar_kkt_rms_hu": kkt,
            "relaxed_M_vs_unrelaxed_2M": pairs, "proposed_vs_simple_relaxation": algs,
            "majorizers": majorizers}
    print(json.dumps(line), flush=True)
    return 0


def fov_mask_np(g):
    """Pixel centres inside the field-of-view disk (the RMSD region)."""
    xc = (np.arange(g.nx) - (g.nx - 1) / 2.0 + g.offset_x) * g.dx
    yc = (np.arange(g.ny) - (g.ny - 1) / 2.0 + g.offset_y) * g.dy
    return (xc[None, :] ** 2 + yc[:, None] ** 2) <= g.fov_radius() ** 2


def kkt_rms_hu(ct, G, g, y, w, x, beta, delta, potential, hu):
    """RMS of [x - D^{-1} grad Psi(x)]_+ - x with D = D_L + D_R, in HU, over the FOV."""
    import torch

    Ax = torch.empty((g.na,) + G.view_shape, device="cuda")
    ct.ct_forward(G, x, Ax)
    r = w * (Ax - y)
    gl = torch.empty_like(x)
    ct.ct_back(G, r, gl)
    gr = torch.empty_like(x)
    cv = torch.empty_like(x)
    ct.ct_reg_gradient(G, x, beta, delta, potential, gr, cv)
    dl = torch.empty_like(x)
    ct.ct_sqs_diag(G, w, dl)
    res = torch.clamp(x - (gl + gr) / (dl + cv), min=0.0) - x
    X = (torch.arange(g.nx, device="cuda") - (g.nx - 1) / 2.0) * g.dx
    Y = (torch.arange(g.ny, device="cuda") - (g.ny - 1) / 2.0) * g.dy
    mask = (X[None, :] ** 2 + Y[:, None] ** 2) <= g.fov_radius() ** 2
    if res.dim() == 3:
        mask = mask.expand(res.shape[0], -1, -1)
    return float(torch.sqrt((res[mask].double() ** 2).mean()) * hu)


def _code_only(src):
    """C++ source without its comments and whitespace (a comment or layout edit keeps the digest)."""
    import re

    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return "".join(src.split())


def _source_digest(csrc=None):
    """Digest of the code of the profiled projector kernels: fp_csr_kernel through bp_records_kernel in
    projectors.cu and the device-arithmetic section of ct_internal.cuh (the functions they inline),
    comments left out."""
    import hashlib

    csrc = csrc or os.path.join(ROOT, "paper_1512_04564_gb300", "csrc")
    h = hashlib.sha256()
    src = open(os.path.join(csrc, "projectors.cu")).read()
    a = src.rfind("template", 0, src.index("fp_csr_kernel(FanDev G"))
    b = src.rfind("template", 0, src.index("bp_fan2d_kernel(FanDev G"))
    h.update(_code_only(src[a:b]).encode())  # fp_csr_kernel .. bp_records_kernel (with bp_epilogue)
    hdr = open(os.path.join(csrc, "ct_internal.cuh")).read()
    a = hdr.index("// ---------------------------------------------------------------- device arithmetic")
    b = hdr.index("// ---------------------------------------------------------------- launchers")
    h.update(_code_only(hdr[a:b]).encode())
    return h.hexdigest()[:16]


# Algorithmic FP32 work of the projector pair, per nonzero a_ij: a footprint evaluation per (pixel, view)
# (four corner fan angles, their sort, the amplitude) spread over the ~3.3 cells it covers, plus each
# cell's trapezoid integral and multiply-add: about 15 operations in 2-D (1.3e10 for the 8.5e8 a_ij of
# the 512x512, 984-view scan), about 8.3 in 3-D (the transaxial footprint is shared by a column's
# voxels: 1e12 for the 1.2e11 a_ij of the 512x512x64 helical scan).
FLOP_PER_AIJ_2D = 1.3e10 / 8.5e8
FLOP_PER_AIJ_3D = 1.0e12 / 1.2e11


def fp32_peak_tflops(clock_mhz):
    """FP32 FMA peak: SMs (from the device) x 128 lanes x 2 FLOP x the SM clock (median under load)."""
    import torch

    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = clock_mhz or 2070.0
    return sms * 128 * 2 * mhz * 1e6 / 1e12, f"{sms} SMs x 128 FP32 lanes x 2 FLOP x {mhz:.0f} MHz"


def fan_cells_view(g, v):
    """Nonzero a_ij of view v of the 2-D fan-beam SF matrix: for every pixel, the detector cells its
    footprint [t0, t3] (corner fan angles) overlaps, clipped to the detector."""
    b = g.betas()[v]
    cb, sb = math.cos(b), math.sin(b)
    xc = (np.arange(g.nx) - (g.nx - 1) / 2.0 + g.offset_x) * g.dx
    yc = (np.arange(g.ny) - (g.ny - 1) / 2.0 + g.offset_y) * g.dy
    X, Y = np.meshgrid(xc, yc)
    taus = []
    for sx in (-0.5, 0.5):
        for sy in (-0.5, 0.5):
            px, py = X + sx * g.dx + g.dso * cb, Y + sy * g.dy + g.dso * sb
            taus.append(np.arctan2(-px * sb + py * cb, px * cb + py * sb) * g.dsd / g.ds + (g.ns - 1) / 2.0 - g.offset_s)
    t0, t3 = np.minimum.reduce(taus), np.maximum.reduce(taus)
    s_lo = np.maximum(np.floor(t0 - 0.5) + 1, 0)
    s_hi = np.minimum(np.ceil(t3 + 0.5) - 1, g.ns - 1)
    return float(np.maximum(s_hi - s_lo + 1, 0).sum())


def kernel_roofline(ct, G, g, M, y, w, x, matrix_bytes, clock_mhz=None):
    """Average device time of one subset forward and back projection (CUDA events on the launching
    stream).  The bound of the projectors is the FP32 ALUs: achieved = FLOP_PER_AIJ_2D x the launch's
    nonzero a_ij (counted on the host) / time, against the FP32 FMA peak at the sampled clock.  Beside it,
    the HBM fraction of the compulsory bytes (image, residual rows) and, with the resident matrix, of the
    stored bytes the kernels stream; the slower kernel is reported as the dominant one."""
    import torch

    views = list(range(M - 1, g.na, M))
    nv = len(views)
    out = torch.empty(nv, g.ns, device="cuda")
    xb = torch.empty_like(x)
    reps = 50
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(5):
            fn()
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps * 1e-3

    # the forward projector on the packed image [x | x^T] (the solver's update kernel writes it; ct_forward
    # would add one packing launch)
    xp = torch.empty(2 * x.numel(), device="cuda")
    ct.ct_pack_image(G, x, xp)
    fp_s = timed(lambda: ct.ct_forward_packed(G, xp, out, views=views))
    bp_s = timed(lambda: ct.ct_back(G, out, xb, views=views))
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks else "fallback 6800 GB/s"
    npix = g.nx * g.ny
    nnz = sum(fan_cells_view(g, v) for v in views)
    flops = FLOP_PER_AIJ_2D * nnz
    peak, peak_src = fp32_peak_tflops(clock_mhz)
    # compulsory bytes: FP reads the image once and writes the subset's rays; BP reads the rays, writes the image
    fp_min = 4 * npix + 4 * nv * g.ns
    bp_min = 4 * nv * g.ns + 4 * npix
    stored = {}
    if matrix_bytes:
        R = g.na * g.ns
        # the rows' entries (6 B each: a_ij + 16-bit offset) and chunk bases (4 B per 32 entries)
        _, rec_bytes = ct.ct_geom_matrix_info(G)
        entry_bytes = matrix_bytes - 8 * (R + 1) - 4 * (R + 3) - rec_bytes
        # FP: the subset's share of the entries, 12 B per ray (row and chunk pointers), image, output
        stored["fp"] = entry_bytes * nv / g.na + 12 * nv * g.ns + 4 * npix + 4 * nv * g.ns
        # BP: the subset's share of the records (per view and 32 pixels: a chunk of 16-bit first cells and
        # counts and K weights per pixel; its 4-byte word), the residual rows, x written
        stored["bp"] = rec_bytes * nv / g.na + 4 * nv * g.ns + 4 * npix
    kernels = {}
    for key, t, name, cmin in (("fp", fp_s, "fp_csr_kernel" if matrix_bytes else "fp_bundle_kernel", fp_min),
                               ("bp", bp_s, "bp_records_kernel" if matrix_bytes else "bp_fan2d_kernel", bp_min)):
        k = {"kernel": name, "ms": t * 1e3, "tflops": flops / t / 1e12, "alu_frac": flops / t / 1e12 / peak,
             "compulsory_bytes": cmin, "compulsory_gbs": cmin / t / 1e9, "compulsory_frac": cmin / t / 1e9 / hbm_peak}
        if key in stored:
            k.update({"stored_bytes": stored[key], "stored_gbs": stored[key] / t / 1e9,
                      "stored_frac": stored[key] / t / 1e9 / hbm_peak})
        kernels[key] = k
    dom = "bp" if bp_s >= fp_s else "fp"
    traffic = None
    try:
        tr = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
        if tr.get("source_digest") == _source_digest() and tr.get("views_per_launch") == nv and matrix_bytes:
            traffic = tr["kernels"][dom]["dram_bytes_per_launch"]
    except (OSError, KeyError, ValueError):
        pass
    k = kernels[dom]
    return {
        "bound": "alu", "kernel": k["kernel"] + f" ({nv} views)", "achieved": k["tflops"], "peak": peak,
        "unit": "TFLOP/s", "frac": k["tflops"] / peak, "traffic": traffic,
        "peak_source": peak_src + " (derived from unit counts and the sampled clock)",
        "flop_per_launch": flops, "nnz_per_launch": nnz, "flop_per_aij": FLOP_PER_AIJ_2D,
        "hbm_compulsory": {"bytes": k["compulsory_bytes"], "achieved": k["compulsory_gbs"], "peak": hbm_peak,
                           "unit": "GB/s", "frac": k["compulsory_frac"], "peak_source": hbm_src},
        "hbm_stored": ({"bytes": k["stored_bytes"], "achieved": k["stored_gbs"], "peak": hbm_peak, "unit": "GB/s",
                        "frac": k["stored_frac"], "peak_source": hbm_src} if "stored_bytes" in k else None),
        "views_per_launch": nv, "kernels": kernels,
    }


if __name__ == "__main__":
    sys.exit(main())
