"""Batched relaxed OS-LALM against the single-slice solver and the oracle: slices of several geometries on
concurrent lanes of the single-slice solver, and the slices of one geometry (its large slices one after
another, its small ones in one persistent launch).

A batch mixes image sizes, detector sizes, view counts and subset counts;
some slices use the resident system matrix and some the on-the-fly
footprints; two slices share one geometry.  Each slice must match the
single-slice solve (RMSD <= 0.01 HU: the same arithmetic with a different
summation order in the projectors) and one slice the FP64 oracle
(<= 0.1 HU, the solver parity bar).
"""

import numpy as np
import pytest
import torch

import synth
from oracle import solver as osolver
from oracle.projector import FanProjector

pytestmark = pytest.mark.gpu

MU_W = 0.02
BETA = 2.0 ** 14 / MU_W ** 2
DELTA = 10 * MU_W / 1000
HU = 1000 / MU_W


def _problem(seed, nx, ns, na, dx):
    g = synth.FanArcGeometry(nx=nx, ny=nx, dx=dx, dy=dx, ns=ns, ds=1.0239 * 128 / ns * nx * dx / 128, na=na,
                             dso=541.0, dsd=949.0)
    r = 0.4 * nx * dx
    E = [synth.Ellipse(0.0, 0.0, r, 0.8 * r, 0.2 + seed, 0.018), synth.Ellipse(0.2 * r, -0.1 * r, 0.2 * r, 0.15 * r, 0.0, -0.01),
         synth.Ellipse(-0.3 * r, 0.2 * r, 0.1 * r, 0.1 * r, 0.0, 0.006)]
    y, w = synth.transmission_data(synth.fan_arc_line_integrals(E, g), 1e5, 5.0, seed)
    return g, y.astype(np.float32), w.astype(np.float32)


CASES = [  # (seed, nx, ns, na, dx, M, resident)
    (1, 64, 96, 90, 2.0, 5, True),
    (2, 96, 128, 120, 1.4, 12, False),
    (3, 128, 160, 180, 1.0, 10, True),
    (4, 64, 96, 90, 2.0, 9, True),     # shares the first slice's geometry
    (5, 80, 112, 60, 1.6, 7, False),   # uneven subsets (60 = 7 * 8 + 4)
]


def _hu_rmsd(a, b, g):
    return osolver.rmsd_hu(a.astype(np.float64), b.astype(np.float64), osolver.fov_mask(g), HU)


def test_batched_matches_single_slice_solves():
    from paper_1512_04564_gb300 import ct

    geoms, ys, ws, xs, params, probs = {}, [], [], [], [], []
    for seed, nx, ns, na, dx, M, resident in CASES:
        key = (nx, ns, na, dx)
        g, y, w = _problem(seed, nx, ns, na, dx)
        if key not in geoms:
            G = ct.Geometry.from_fan(g)
            if resident:
                ct.ct_geom_precompute(G)
            geoms[key] = G
        probs.append((g, geoms[key], y, w, M))
        ys.append(torch.from_numpy(y).cuda())
        ws.append(torch.from_numpy(w).cuda())
        xs.append(torch.zeros(g.ny, g.nx, device="cuda"))
        params.append(dict(M=M, n_iter=4, alpha=1.999, beta=BETA, delta=DELTA))
    G_list = [p[1] for p in probs]
    # references: one single-slice solve per slice, also its x* for the trace
    singles, refs = [], []
    for i, (g, G, y, w, M) in enumerate(probs):
        xr = torch.zeros(g.ny, g.nx, device="cuda")
        ct.ct_relaxed_oslalm_solve(G, ys[i], ws[i], xr, M=1, n_iter=30, alpha=1.999, beta=BETA, delta=DELTA)
        refs.append(xr)
        xsng = torch.zeros(g.ny, g.nx, device="cuda")
        rep = ct.ct_relaxed_oslalm_solve(G, ys[i], ws[i], xsng, x_ref=xr, hu_per_unit=HU, **params[i])
        singles.append((xsng, rep))
        params[i]["x_ref"] = xr
        params[i]["hu_per_unit"] = HU
    reps = ct.ct_relaxed_oslalm_solve_batched(G_list, ys, ws, xs, params)
    torch.cuda.synchronize()
    for i, (g, G, y, w, M) in enumerate(probs):
        d = _hu_rmsd(xs[i].cpu().numpy(), singles[i][0].cpu().numpy(), g)
        assert d <= 0.01, (i, d)
        tb, ts = reps[i]["rmsd_trace_hu"], singles[i][1]["rmsd_trace_hu"]
        assert len(tb) == 4 and np.allclose(tb, ts, rtol=1e-3, atol=1e-2), (i, tb, ts)
        assert all(b > a for a, b in zip(reps[i]["iter_seconds"], reps[i]["iter_seconds"][1:]))


def test_large_slices_of_one_geometry_solved_one_after_another():
    """Slices of >= 384 x 384 pixels run the single-slice solver inside the batched call; slices of one
    geometry share its workspace, so they are solved one after the other: each result is the single
    solve's, bit for bit, and the second slice's iterations start after the first's end."""
    from paper_1512_04564_gb300 import ct

    probs = [_problem(6, 384, 400, 72, 0.5), _problem(10, 384, 400, 72, 0.5)]
    G = ct.Geometry.from_fan(probs[0][0])
    ys = [torch.from_numpy(p[1]).cuda() for p in probs]
    ws = [torch.from_numpy(p[2]).cuda() for p in probs]
    params, singles = [], []
    for i, (g, _, _) in enumerate(probs):
        xr = torch.zeros(g.ny, g.nx, device="cuda")
        ct.ct_relaxed_oslalm_solve(G, ys[i], ws[i], xr, M=1, n_iter=20, alpha=1.999, beta=BETA, delta=DELTA)
        p = dict(M=6, n_iter=3, alpha=1.999, beta=BETA, delta=DELTA, x_ref=xr, hu_per_unit=HU)
        xs = torch.zeros(g.ny, g.nx, device="cuda")
        singles.append((xs, ct.ct_relaxed_oslalm_solve(G, ys[i], ws[i], xs, **p)))
        params.append(p)
    xb = [torch.zeros(p[0].ny, p[0].nx, device="cuda") for p in probs]
    reps = ct.ct_relaxed_oslalm_solve_batched([G, G], ys, ws, xb, params)
    torch.cuda.synchronize()
    for i in range(2):
        assert torch.equal(xb[i], singles[i][0]), i
        assert len(reps[i]["rmsd_trace_hu"]) == 3 and reps[i]["rmsd_trace_hu"][-1] < reps[i]["rmsd_trace_hu"][0]
        assert all(b > a for a, b in zip(reps[i]["iter_seconds"], reps[i]["iter_seconds"][1:]))
    assert reps[0]["seconds"] == reps[1]["seconds"]
    assert reps[0]["iter_seconds"][-1] <= reps[1]["iter_seconds"][0]
    assert reps[1]["iter_seconds"][-1] <= reps[1]["seconds"] * (1 + 1e-6)


def test_persistent_launch_matches_single_slice_solves():
    """Small slices of one geometry share one persistent launch (different data and subset counts): each
    matches its single-slice solve (RMSD <= 0.01 HU: the same arithmetic with a different summation order
    in the projectors), the traces too."""
    from paper_1512_04564_gb300 import ct

    g0 = _problem(1, 64, 96, 90, 2.0)[0]
    G = ct.Geometry.from_fan(g0)
    ct.ct_geom_precompute(G)
    probs = [_problem(seed, 64, 96, 90, 2.0) for seed in (1, 4, 9)]
    Ms = (5, 9, 7)
    ys = [torch.from_numpy(p[1]).cuda() for p in probs]
    ws = [torch.from_numpy(p[2]).cuda() for p in probs]
    params, singles = [], []
    for i, (g, _, _) in enumerate(probs):
        xr = torch.zeros(g.ny, g.nx, device="cuda")
        ct.ct_relaxed_oslalm_solve(G, ys[i], ws[i], xr, M=1, n_iter=30, alpha=1.999, beta=BETA, delta=DELTA)
        p = dict(M=Ms[i], n_iter=4, alpha=1.999, beta=BETA, delta=DELTA, x_ref=xr, hu_per_unit=HU)
        xs = torch.zeros(g.ny, g.nx, device="cuda")
        singles.append((xs, ct.ct_relaxed_oslalm_solve(G, ys[i], ws[i], xs, **p)))
        params.append(p)
    xb = [torch.zeros(g0.ny, g0.nx, device="cuda") for _ in probs]
    reps = ct.ct_relaxed_oslalm_solve_batched([G] * 3, ys, ws, xb, params)
    torch.cuda.synchronize()
    for i, (g, _, _) in enumerate(probs):
        d = _hu_rmsd(xb[i].cpu().numpy(), singles[i][0].cpu().numpy(), g)
        assert d <= 0.01, (i, d)
        tb, ts = reps[i]["rmsd_trace_hu"], singles[i][1]["rmsd_trace_hu"]
        assert len(tb) == 4 and np.allclose(tb, ts, rtol=1e-3, atol=1e-2), (i, tb, ts)


def test_large_slices_of_several_geometries_run_concurrently():
    """Large slices of different geometries are solved by the single-slice solver on concurrent streams
    (one geometry's slices one after another, as they share its workspace): each result is the single
    solve's, bit for bit, and each slice's times count from the call's start and stay within its total."""
    from paper_1512_04564_gb300 import ct

    probs = [_problem(6, 384, 400, 72, 0.5), _problem(7, 384, 320, 60, 0.55), _problem(8, 384, 400, 72, 0.5)]
    Gs = [ct.Geometry.from_fan(probs[0][0]), ct.Geometry.from_fan(probs[1][0])]
    G_of = [Gs[0], Gs[1], Gs[0]]  # the third slice shares the first one's geometry
    ys = [torch.from_numpy(p[1]).cuda() for p in probs]
    ws = [torch.from_numpy(p[2]).cuda() for p in probs]
    params, singles = [], []
    for i, (g, _, _) in enumerate(probs):
        xr = torch.zeros(g.ny, g.nx, device="cuda")
        ct.ct_relaxed_oslalm_solve(G_of[i], ys[i], ws[i], xr, M=1, n_iter=10, alpha=1.999, beta=BETA, delta=DELTA)
        p = dict(M=6, n_iter=3, alpha=1.999, beta=BETA, delta=DELTA, x_ref=xr, hu_per_unit=HU)
        xs = torch.zeros(g.ny, g.nx, device="cuda")
        singles.append((xs, ct.ct_relaxed_oslalm_solve(G_of[i], ys[i], ws[i], xs, **p)))
        params.append(p)
    xb = [torch.zeros(p[0].ny, p[0].nx, device="cuda") for p in probs]
    reps = ct.ct_relaxed_oslalm_solve_batched(G_of, ys, ws, xb, params)
    torch.cuda.synchronize()
    for i in range(3):
        assert torch.equal(xb[i], singles[i][0]), i
        assert reps[i]["rmsd_trace_hu"] == singles[i][1]["rmsd_trace_hu"], i
        t = reps[i]["iter_seconds"]
        assert len(t) == 3 and 0 < t[0] < t[1] < t[2] <= reps[i]["seconds"] * (1 + 1e-6), (i, t)
        assert reps[i]["seconds"] == reps[0]["seconds"]
    # the two slices of one geometry ran one after the other
    assert reps[0]["iter_seconds"][-1] <= reps[2]["iter_seconds"][0] or reps[2]["iter_seconds"][-1] <= reps[0]["iter_seconds"][0]


def test_batched_slice_matches_oracle():
    from paper_1512_04564_gb300 import ct

    seed, nx, ns, na, dx, M, _ = CASES[2]
    g, y, w = _problem(seed, nx, ns, na, dx)
    G = ct.Geometry.from_fan(g)
    seed2, nx2, ns2, na2, dx2, M2, _ = CASES[0]
    g2, y2, w2 = _problem(seed2, nx2, ns2, na2, dx2)
    G2 = ct.Geometry.from_fan(g2)
    x1 = torch.zeros(g.ny, g.nx, device="cuda")
    x2 = torch.zeros(g2.ny, g2.nx, device="cuda")
    p = dict(n_iter=3, alpha=1.999, beta=BETA, delta=DELTA)
    ct.ct_relaxed_oslalm_solve_batched([G, G2], [torch.from_numpy(y).cuda(), torch.from_numpy(y2).cuda()],
                                       [torch.from_numpy(w).cuda(), torch.from_numpy(w2).cuda()], [x1, x2],
                                       [dict(M=M, **p), dict(M=M2, **p)])
    prob = osolver.PWLSProblem(FanProjector(g), y.astype(np.float64), w.astype(np.float64), BETA, DELTA)
    xo = osolver.relaxed_os_lalm(prob, np.zeros((g.ny, g.nx)), M, 1.999, 3)
    assert _hu_rmsd(x1.cpu().numpy(), xo, g) <= 0.1


def test_batched_rejects_bad_arguments():
    from paper_1512_04564_gb300 import ct

    g, y, w = _problem(*CASES[0][:5])
    G = ct.Geometry.from_fan(g)
    with pytest.raises(ct.CTError):
        ct.ct_relaxed_oslalm_solve_batched([G], [torch.from_numpy(y).cuda()], [torch.from_numpy(w).cuda()],
                                           [torch.zeros(g.ny, g.nx, device="cuda")],
                                           [dict(M=0, n_iter=2, alpha=1.999, beta=BETA, delta=DELTA)])


def test_autotune_choice_keeps_parity():
    from paper_1512_04564_gb300 import ct

    g, y, w = _problem(*CASES[2][:5])
    G = ct.Geometry.from_fan(g)
    ct.ct_geom_precompute(G)
    fp, bp = ct.ct_geom_autotune(G, 20)
    assert fp in ("resident rows", "bundle", "ray") and bp in ("stored footprints", "on the fly")
    x = torch.from_numpy(np.random.default_rng(0).random((g.ny, g.nx)).astype(np.float32)).cuda()
    yy = torch.empty(g.na, g.ns, device="cuda")
    ct.ct_forward(G, x, yy)
    ref = FanProjector(g).forward(x.cpu().numpy().astype(np.float64))
    den = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    assert np.max(np.abs(yy.cpu().numpy() - ref) / den) <= 1e-5


def test_grid_barrier_wait_runs_out_and_context_survives():
    """Failure detection of the persistent launch: with a barrier participant that never arrives and a
    short poll limit, every grid-barrier wait gives up, the call returns CT_ETIMEOUT, and the next
    call on the same context (hook reset) solves normally and matches a solve made before the failure."""
    from paper_1512_04564_gb300 import ct

    g, y, w = _problem(*CASES[0][:5])
    G = ct.Geometry.from_fan(g)
    yd, wd = torch.from_numpy(y).cuda(), torch.from_numpy(w).cuda()
    p = dict(M=5, n_iter=2, alpha=1.999, beta=BETA, delta=DELTA)
    x_ok = torch.zeros(g.ny, g.nx, device="cuda")
    ct.ct_relaxed_oslalm_solve_batched([G], [yd], [wd], [x_ok], [p])
    try:
        ct.ct_debug_barrier(max_polls=2000, missing=1)
        x_bad = torch.zeros(g.ny, g.nx, device="cuda")
        with pytest.raises(ct.CTError) as e:
            ct.ct_relaxed_oslalm_solve_batched([G], [yd], [wd], [x_bad], [p])
        assert e.value.status == ct.CT_ETIMEOUT
        assert "barrier" in str(e.value)
    finally:
        ct.ct_debug_barrier(0, 0)
    x2 = torch.zeros(g.ny, g.nx, device="cuda")
    ct.ct_relaxed_oslalm_solve_batched([G], [yd], [wd], [x2], [p])
    torch.cuda.synchronize()
    assert _hu_rmsd(x2.cpu().numpy(), x_ok.cpu().numpy(), g) <= 1e-6
    with pytest.raises(ct.CTError) as e:
        ct.ct_debug_barrier(-1, 0)
    assert e.value.status == ct.CT_EINVAL


def test_batched_slices_stop_at_their_tolerance():
    """With x_ref and stop_rmsd_hu each slice leaves the persistent launch at the end of its first outer
    iteration at the tolerance, as the single-slice solver stops: same iteration count, same image."""
    from paper_1512_04564_gb300 import ct

    probs, Gs = [], {}
    for seed, nx, ns, na, dx, M, resident in CASES:
        key = (nx, ns, na, dx)
        g, y, w = _problem(seed, nx, ns, na, dx)
        if key not in Gs:
            Gs[key] = ct.Geometry.from_fan(g)
            if resident:
                ct.ct_geom_precompute(Gs[key])
        probs.append((g, Gs[key], torch.from_numpy(y).cuda(), torch.from_numpy(w).cuda(), M))
    refs, params, singles = [], [], []
    for g, G, y, w, M in probs:
        xr = torch.zeros(g.ny, g.nx, device="cuda")
        ct.ct_relaxed_oslalm_solve(G, y, w, xr, M=1, n_iter=30, alpha=1.999, beta=BETA, delta=DELTA)
        # a tolerance each slice first meets at iteration 3: between its single-slice RMSD after iterations
        # 2 and 3 (far from both, so both solvers stop at the same iteration)
        x0 = torch.zeros(g.ny, g.nx, device="cuda")
        tr = ct.ct_relaxed_oslalm_solve(G, y, w, x0, M=M, n_iter=12, alpha=1.999, beta=BETA, delta=DELTA, x_ref=xr,
                                        hu_per_unit=HU)["rmsd_trace_hu"]
        assert tr[0] > tr[1] > tr[2] + 0.1, tr[:3]
        tol = 0.5 * (tr[1] + tr[2])
        p = dict(M=M, n_iter=12, alpha=1.999, beta=BETA, delta=DELTA, x_ref=xr, hu_per_unit=HU, stop_rmsd_hu=tol)
        xs = torch.zeros(g.ny, g.nx, device="cuda")
        singles.append((xs, ct.ct_relaxed_oslalm_solve(G, y, w, xs, **p)))
        params.append(p)
    xb = [torch.zeros(g.ny, g.nx, device="cuda") for g, *_ in probs]
    # one batched call per geometry: the slices of one geometry share the persistent launch
    reps = [None] * len(probs)
    for G in {id(p[1]): p[1] for p in probs}.values():
        idx = [i for i, p in enumerate(probs) if p[1] is G]
        got = ct.ct_relaxed_oslalm_solve_batched([G] * len(idx), [probs[i][2] for i in idx],
                                                 [probs[i][3] for i in idx], [xb[i] for i in idx],
                                                 [params[i] for i in idx])
        for i, r in zip(idx, got):
            reps[i] = r
    torch.cuda.synchronize()
    for i, (g, *_rest) in enumerate(probs):
        xs, rs = singles[i]
        assert rs["iters_done"] == 3
        assert reps[i]["iters_done"] == 3, (i, reps[i]["iters_done"])
        assert reps[i]["rmsd_trace_hu"][-1] <= params[i]["stop_rmsd_hu"] and reps[i]["seconds_to_tol"] > 0
        assert _hu_rmsd(xb[i].cpu().numpy(), xs.cpu().numpy(), g) <= 0.01, i
