"""GPU parity of the helical projector pair with the trapezoid axial footprint (SF-TT).

The kernels run the rectangle model's arithmetic at the ramps' centre and add
the ramp corrections at the row boundaries the ramps straddle; the oracle
integrates each voxel's trapezoid over each row directly.  Same tolerances as
the rectangle model (per ray / per voxel 1e-5 of max(|value|, 1e-3 max), also
for uniform-random volumes reaching the border), on the same four
geometries, plus adjointness, view subsets, D_L, the solver (<= 0.1 HU after
3 iterations of M = 8) and sampled rays and voxels of one subset of the
full 512 x 512 x 64, 2952-view scan.
"""

import dataclasses

import numpy as np
import pytest
import torch

import synth
from oracle import solver as osolver
from oracle.helical import HelicalProjector
from test_gpu_helical import CASES, HU, MU_W, TOL, TOL_BORDER, dev, phantom_volume, rel_err

pytestmark = pytest.mark.gpu

TT_CASES = {k: dataclasses.replace(g, axial="trap") for k, g in CASES.items()}


@pytest.fixture(scope="module")
def ct():
    from paper_1512_04564_gb300 import ct as ctmod

    return ctmod


@pytest.mark.parametrize("case", list(TT_CASES))
@pytest.mark.parametrize("kind", ["phantom", "random"])
def test_forward_parity(ct, case, kind):
    g = TT_CASES[case]
    x = phantom_volume(g) if kind == "phantom" else np.random.default_rng(1).random((g.nz, g.ny, g.nx)).astype(
        np.float32)
    G = ct.Geometry.from_helix(g)
    y = torch.empty(g.na, g.nt, g.ns, device="cuda")
    ct.ct_forward(G, dev(x), y)
    ref = HelicalProjector(g).forward(x.astype(np.float64))
    assert rel_err(y.cpu().numpy(), ref) <= (TOL if kind == "phantom" else TOL_BORDER)
    # and the model is not the rectangle one (except where one voxel spans the whole detector row)
    if case != "one_row":
        rr = HelicalProjector(CASES[case]).forward(x.astype(np.float64))
        assert rel_err(rr, ref) > 3 * (TOL if kind == "phantom" else TOL_BORDER)


@pytest.mark.parametrize("case", list(TT_CASES))
def test_back_parity(ct, case):
    g = TT_CASES[case]
    yv = np.random.default_rng(2).random((g.na, g.nt, g.ns)).astype(np.float32)
    G = ct.Geometry.from_helix(g)
    x = torch.empty(g.nz, g.ny, g.nx, device="cuda")
    ct.ct_back(G, dev(yv), x)
    ref = HelicalProjector(g).back(yv.astype(np.float64))
    assert rel_err(x.cpu().numpy(), ref) <= TOL


def test_adjoint_and_subsets(ct):
    g = TT_CASES["small"]
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
    views = [5, 0, 33, 17, 59]
    P = HelicalProjector(g)
    y = torch.empty(len(views), g.nt, g.ns, device="cuda")
    xp = phantom_volume(g, 1)
    ct.ct_forward(G, dev(xp), y, views=views)
    assert rel_err(y.cpu().numpy(), P.forward(xp.astype(np.float64), views)) <= TOL
    ys = rng.random((len(views), g.nt, g.ns)).astype(np.float32)
    x0 = rng.random((g.nz, g.ny, g.nx)).astype(np.float32)
    xo = dev(x0)
    ct.ct_back(G, dev(ys), xo, views=views, scale=-0.5, accumulate=True)
    ref = x0.astype(np.float64) - 0.5 * P.back(ys.astype(np.float64), views)
    np.testing.assert_allclose(xo.cpu().numpy(), ref, rtol=2e-5, atol=2e-5 * np.abs(ref).max())


def test_sqs_diag_parity(ct):
    g = TT_CASES["small"]
    w = np.random.default_rng(5).uniform(10.0, 1e4, (g.na, g.nt, g.ns)).astype(np.float32)
    G = ct.Geometry.from_helix(g)
    d = torch.empty(g.nz, g.ny, g.nx, device="cuda")
    ct.ct_sqs_diag(G, dev(w), d)
    P = HelicalProjector(g)
    ref = P.back(w.astype(np.float64) * P.forward(np.ones(P.shape)))
    assert rel_err(d.cpu().numpy(), ref) <= TOL


def test_solver_matches_oracle(ct):
    g = dataclasses.replace(synth.helix3d_64().geom, axial="trap")
    S = synth.phantom_of(synth.helix3d_64(0))
    y, w = synth.transmission_data(synth.helical_line_integrals(S, g, n_sub=2), 1e5, 5.0, 0)
    y, w = y.astype(np.float32), w.astype(np.float32)
    beta = 2.0 ** 14 / MU_W ** 2
    delta = 10 * MU_W / 1000
    M, n_iter = 8, 3
    G = ct.Geometry.from_helix(g)
    x = torch.zeros(g.nz, g.ny, g.nx, device="cuda")
    ct.ct_relaxed_oslalm_solve(G, dev(y), dev(w), x, M=M, n_iter=n_iter, alpha=1.999, beta=beta, delta=delta)
    prob = osolver.PWLSProblem(HelicalProjector(g), y.astype(np.float64), w.astype(np.float64), beta, delta)
    xo = osolver.relaxed_os_lalm(prob, np.zeros((g.nz, g.ny, g.nx)), M, 1.999, n_iter)
    d = osolver.rmsd_hu(x.cpu().numpy().astype(np.float64), xo, osolver.fov_mask(g), HU)
    assert d <= 0.1, d


def test_full_size_sampled(ct):
    cfg = synth.helix3d_512()
    g = dataclasses.replace(cfg.geom, axial="trap")
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
    yv = rng.random((len(views), g.nt, g.ns)).astype(np.float32)
    xb = torch.empty(g.nz, g.ny, g.nx, device="cuda")
    ct.ct_back(G, dev(yv), xb, views=views.tolist())
    vox = rng.integers(0, g.nx * g.ny * g.nz, 64)
    refb = P.back_voxels(yv.astype(np.float64), views, vox)
    got = xb.cpu().numpy().reshape(-1)[vox]
    den = np.maximum(np.abs(refb), 1e-3 * np.abs(xb.cpu().numpy()).max())
    assert np.max(np.abs(got - refb) / den) <= TOL
