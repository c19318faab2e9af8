"""GPU parity of the helical cone-beam path (SF-TR projector pair, 26-neighbour regularizer,
relaxed OS-LALM) against the FP64 oracle, through the C ABI.

Tolerances follow the 2-D path's: per ray / per voxel |gpu - oracle| <= 1e-5 x
max(|oracle|, 1e-3 max|oracle|), for volumes shaped like the workloads and for
uniform-random volumes whose signal reaches the border (sliver-thin transaxial
footprint overlaps; the transaxial footprint is the 2-D one, whose vertices
are placed to about 1e-7 cells); <A x, y> vs <x, A'y> from the GPU
outputs to 1e-5; the solver within 0.1 HU RMSD after a fixed iteration count.
The axial footprint adds no tighter limit: its row boundaries are placed to
about 4e-6 of a voxel (FP32 coordinates up to ~100 voxels), which moves at
most that fraction of one voxel's value between adjacent rows.
"""

import numpy as np
import pytest
import torch

import synth
from oracle import regularizer as oreg
from oracle import solver as osolver
from oracle.helical import HelicalProjector

pytestmark = pytest.mark.gpu

TOL = 1e-5
TOL_BORDER = TOL
MU_W = 0.02
HU = 1000.0 / MU_W


def small(**kw):
    base = dict(nx=40, ny=36, nz=20, dx=2.0, dy=2.2, dz=1.0, ns=72, ds=2.0, nt=8, dt=2.4, na=60, dso=300.0,
                dsd=520.0, pitch=0.8, orbit_deg=720.0, orbit_start_deg=7.0, offset_x=0.3, offset_y=-0.2,
                offset_z=0.1, offset_s=0.25, offset_t=-0.15)
    base.update(kw)
    return synth.HelicalConeGeometry(**base)


CASES = {
    "small": small(),
    "rows20": small(nt=20, dt=1.1, nz=33, dz=0.7, na=48),   # 32-row variant, three ragged chunks
    "one_row": small(nt=1, nz=1, dz=30.0, pitch=0.0, offset_z=0.0, offset_t=0.0, na=36),
    "helix3d_64": synth.helix3d_64().geom,
}


@pytest.fixture(scope="module")
def ct():
    from paper_1512_04564_gb300 import ct as ctmod

    return ctmod


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    return float(np.max(np.abs(got - ref) / den))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def phantom_volume(g, seed=0, oversample=2):
    rng = np.random.default_rng(seed)
    r = 0.4 * min(g.nx * g.dx, g.ny * g.dy)
    zh = 0.45 * g.nz * g.dz
    S = [synth.EllipticCylinder(0.0, 0.0, r, 0.9 * r, 0.3, -zh, zh, 0.015)]
    for _ in range(5):
        S.append(synth.Ellipsoid(rng.uniform(-0.4, 0.4) * r, rng.uniform(-0.4, 0.4) * r, rng.uniform(-0.5, 0.5) * zh,
                                 rng.uniform(0.1, 0.3) * r, rng.uniform(0.1, 0.3) * r, rng.uniform(0.2, 0.5) * zh,
                                 rng.uniform(0, 3), rng.uniform(-0.005, 0.005)))
    return synth.rasterize_solids(S, g, oversample=oversample, oversample_z=oversample).astype(np.float32)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("kind", ["phantom", "random"])
def test_forward_parity(ct, case, kind):
    g = CASES[case]
    x = phantom_volume(g) if kind == "phantom" else np.random.default_rng(1).random((g.nz, g.ny, g.nx)).astype(
        np.float32)
    G = ct.Geometry.from_helix(g)
    y = torch.empty(g.na, g.nt, g.ns, device="cuda")
    ct.ct_forward(G, dev(x), y)
    ref = HelicalProjector(g).forward(x.astype(np.float64))
    e = rel_err(y.cpu().numpy(), ref)
    print(f"helical forward {case} {kind}: worst per-ray error {e:.2e}")
    assert e <= (TOL if kind == "phantom" else TOL_BORDER)


@pytest.mark.parametrize("case", list(CASES))
def test_back_parity(ct, case):
    g = CASES[case]
    yv = np.random.default_rng(2).random((g.na, g.nt, g.ns)).astype(np.float32)
    G = ct.Geometry.from_helix(g)
    x = torch.empty(g.nz, g.ny, g.nx, device="cuda")
    ct.ct_back(G, dev(yv), x)
    ref = HelicalProjector(g).back(yv.astype(np.float64))
    assert rel_err(x.cpu().numpy(), ref) <= TOL


def test_adjoint_pair(ct):
    g = CASES["small"]
    rng = np.random.default_rng(3)
    x = rng.random((g.nz, g.ny, g.nx)).astype(np.float32)
    yv = rng.random((g.na, g.nt, g.ns)).astype(np.float32)
    G = ct.Geometry.from_helix(g)
    Ax = torch.empty(g.na, g.nt, g.ns, device="cuda")
    Aty = torch.empty(g.nz, g.ny, g.nx, device="cuda")
    ct.ct_forward(G, dev(x), Ax)
    ct.ct_back(G, dev(yv), Aty)
    lhs = float(np.sum(Ax.cpu().numpy().astype(np.float64) * yv))
    rhs = float(np.sum(x.astype(np.float64) * Aty.cpu().numpy()))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_view_subsets_scale_and_accumulate(ct):
    g = CASES["small"]
    views = [5, 0, 33, 17, 59]
    rng = np.random.default_rng(4)
    x = phantom_volume(g, 1)
    G = ct.Geometry.from_helix(g)
    P = HelicalProjector(g)
    y = torch.empty(len(views), g.nt, g.ns, device="cuda")
    ct.ct_forward(G, dev(x), y, views=views)
    assert rel_err(y.cpu().numpy(), P.forward(x.astype(np.float64), views)) <= TOL
    yv = rng.random((len(views), g.nt, g.ns)).astype(np.float32)
    x0 = rng.random((g.nz, g.ny, g.nx)).astype(np.float32)
    xo = dev(x0)
    ct.ct_back(G, dev(yv), xo, views=views, scale=-0.5, accumulate=True)
    ref = x0.astype(np.float64) - 0.5 * P.back(yv.astype(np.float64), views)
    np.testing.assert_allclose(xo.cpu().numpy(), ref, rtol=2e-5, atol=2e-5 * np.abs(ref).max())


def test_sqs_diag_parity(ct):
    g = CASES["small"]
    w = np.random.default_rng(5).uniform(10.0, 1e4, (g.na, g.nt, g.ns)).astype(np.float32)
    G = ct.Geometry.from_helix(g)
    d = torch.empty(g.nz, g.ny, g.nx, device="cuda")
    ct.ct_sqs_diag(G, dev(w), d)
    P = HelicalProjector(g)
    ref = P.back(w.astype(np.float64) * P.forward(np.ones(P.shape)))
    assert rel_err(d.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("pot", ["hyperbola", "fair", "quadratic"])
def test_regularizer_26_neighbours(ct, pot):
    g = small(nx=37, ny=29, nz=11)
    x = np.random.default_rng(6).random((g.nz, g.ny, g.nx)).astype(np.float32) * 0.02
    G = ct.Geometry.from_helix(g)
    gr = torch.empty(g.nz, g.ny, g.nx, device="cuda")
    cv = torch.empty_like(gr)
    beta, delta = 3.0, 2e-4
    ct.ct_reg_gradient(G, dev(x), beta, delta, pot, gr, cv)
    x64 = x.astype(np.float64)
    rg = oreg.gradient(x64, beta, delta, pot)
    rc = oreg.curvature(x64, beta, delta, pot)
    assert np.max(np.abs(gr.cpu().numpy() - rg)) <= 1e-5 * np.abs(rg).max()
    assert rel_err(cv.cpu().numpy(), rc) <= 1e-5


def _problem(g, seed=0):
    S = synth.phantom_of(synth.helix3d_64(seed))
    li = synth.helical_line_integrals(S, g, n_sub=2)
    y, w = synth.transmission_data(li, 1e5, 5.0, seed)
    return y.astype(np.float32), w.astype(np.float32)


@pytest.mark.parametrize("algorithm", ["proposed", "simple"])
def test_solver_matches_oracle(ct, algorithm):
    g = synth.helix3d_64().geom
    y, w = _problem(g)
    beta = 2.0 ** 14 / MU_W ** 2
    delta = 10 * MU_W / 1000
    M, n_iter = 8, 3
    G = ct.Geometry.from_helix(g)
    x = torch.zeros(g.nz, g.ny, g.nx, device="cuda")
    rep = ct.ct_relaxed_oslalm_solve(G, dev(y), dev(w), x, M=M, n_iter=n_iter, alpha=1.999, beta=beta, delta=delta,
                                     algorithm=algorithm)
    assert rep["iters_done"] == n_iter
    prob = osolver.PWLSProblem(HelicalProjector(g), y.astype(np.float64), w.astype(np.float64), beta, delta)
    xo = osolver.relaxed_os_lalm(prob, np.zeros((g.nz, g.ny, g.nx)), M, 1.999, n_iter, algorithm=algorithm)
    mask = osolver.fov_mask(g)
    d = osolver.rmsd_hu(x.cpu().numpy().astype(np.float64), xo, mask, HU)
    assert d <= 0.1, d
    # and the iterate moved well away from the start
    assert osolver.rmsd_hu(xo, np.zeros_like(xo), mask, HU) > 100.0


def test_solver_rmsd_trace_against_reference(ct):
    """x_ref and the RMSD trace work on helical volumes (the trace of x* against itself is 0)."""
    g = synth.helix3d_64().geom
    y, w = _problem(g)
    G = ct.Geometry.from_helix(g)
    beta = 2.0 ** 14 / MU_W ** 2
    delta = 10 * MU_W / 1000
    xs = torch.zeros(g.nz, g.ny, g.nx, device="cuda")
    ct.ct_relaxed_oslalm_solve(G, dev(y), dev(w), xs, M=4, n_iter=6, alpha=1.999, beta=beta, delta=delta)
    x = torch.zeros_like(xs)
    rep = ct.ct_relaxed_oslalm_solve(G, dev(y), dev(w), x, M=8, n_iter=3, alpha=1.999, beta=beta, delta=delta,
                                     x_ref=xs, hu_per_unit=HU)
    mask = osolver.fov_mask(g)
    last = osolver.rmsd_hu(x.cpu().numpy().astype(np.float64), xs.cpu().numpy().astype(np.float64), mask, HU)
    assert abs(rep["rmsd_trace_hu"][-1] - last) <= 1e-3 * last + 1e-3


def test_full_size_sampled(ct):
    """512x512x64 voxels, 888x32 cells, 2952 views (three turns): one ordered subset of 123 views
    projected and back-projected on the GPU, sampled rays and voxels computed by the oracle."""
    cfg = synth.helix3d_512()
    g = cfg.geom
    G = ct.Geometry.from_helix(g)
    views = np.arange(5, g.na, cfg.M)
    x = phantom_volume(g, 2, oversample=1)
    y = torch.empty(len(views), g.nt, g.ns, device="cuda")
    ct.ct_forward(G, dev(x), y, views=views.tolist())
    yg = y.cpu().numpy()
    rng = np.random.default_rng(7)
    k = rng.integers(0, len(views), 48)
    rt, rs = rng.integers(0, g.nt, 48), rng.integers(g.ns // 4, 3 * g.ns // 4, 48)
    P = HelicalProjector(g)
    ref = P.forward_rays(x.astype(np.float64), views[k], rt, rs)
    den = np.maximum(np.abs(ref), 1e-3 * np.abs(yg).max())
    assert np.max(np.abs(yg[k, rt, rs] - ref) / den) <= TOL
    # back-projection of the same subset at sampled voxels
    yv = rng.random((len(views), g.nt, g.ns)).astype(np.float32)
    xb = torch.empty(g.nz, g.ny, g.nx, device="cuda")
    ct.ct_back(G, dev(yv), xb, views=views.tolist())
    vox = rng.integers(0, g.nx * g.ny * g.nz, 64)
    refb = P.back_voxels(yv.astype(np.float64), views, vox)
    got = xb.cpu().numpy().reshape(-1)[vox]
    den = np.maximum(np.abs(refb), 1e-3 * np.abs(xb.cpu().numpy()).max())
    assert np.max(np.abs(got - refb) / den) <= TOL


def test_unsupported_calls_on_helical_geometry(ct):
    g = CASES["small"]
    G = ct.Geometry.from_helix(g)
    with pytest.raises(ct.CTError) as e:
        ct.ct_geom_precompute(G)
    assert e.value.status == ct.CT_ENOTSUP
    # the helical start image needs whole turns: less than one turn is refused
    g2 = g.with_(orbit_deg=300.0)
    G2 = ct.Geometry.from_helix(g2)
    y = torch.zeros(g2.na, g2.nt, g2.ns, device="cuda")
    with pytest.raises(ct.CTError) as e:
        ct.ct_fbp(G2, y, torch.zeros(g2.nz, g2.ny, g2.nx, device="cuda"))
    assert e.value.status == ct.CT_ENOTSUP
