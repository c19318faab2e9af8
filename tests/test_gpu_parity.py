"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (from the FP32 arithmetic of the kernels):
* forward projection, per ray: |gpu - oracle| <= 1e-5 * max(|oracle|, 1e-3 max|oracle|),
  for images shaped like the workloads and for uniform-random images whose
  signal reaches the image border, where a ray can take its whole value from
  pixels whose footprints overlap it by slivers of a small fraction of a cell.
  The kernels place each footprint vertex to about 1e-7 cells (an exact FP32
  linear term from FP64-derived anchors, small corrections) and take a cell's
  integral from the nearer end of the trapezoid, so a sliver keeps its
  relative precision;
* back-projection, per pixel: the same rule;
* <A x, y> vs <x, A'y> computed from the GPU outputs: 1e-5 relative;
* relaxed OS-LALM after a fixed iteration count: RMSD(gpu, oracle) <= 0.1 HU.
"""

import numpy as np
import pytest
import torch

import synth
from oracle import regularizer as oreg
from oracle import solver as osolver
from oracle.projector import FanProjector

pytestmark = pytest.mark.gpu

TOL_RAY = 1e-5
SMALL = synth.FanArcGeometry(nx=37, ny=21, dx=1.1, dy=0.9, ns=61, ds=1.3, na=45, dso=200.0, dsd=350.0,
                             offset_x=0.3, offset_y=-0.45, offset_s=0.25, orbit_start_deg=7.0, orbit_deg=300.0)


@pytest.fixture(scope="module")
def ct():
    from paper_1512_04564_gb300 import ct as ctmod

    return ctmod


@pytest.fixture(params=["on_the_fly", "resident_matrix"])
def make_geom(request, ct):
    """Geometry factory for both projector paths: footprints evaluated on the fly, or streamed
    from the resident system matrix built by ct_geom_precompute."""

    def make(g):
        G = ct.Geometry.from_fan(g)
        if request.param == "resident_matrix":
            assert ct.ct_geom_precompute(G) > 0
        return G

    return make


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    return float(np.max(np.abs(got - ref) / den))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def phantom_image(g, seed=0):
    rng = np.random.default_rng(seed)
    E = [synth.Ellipse(0.0, 0.0, 0.42 * g.nx * g.dx, 0.38 * g.ny * g.dy, 0.2, 0.015)]
    for _ in range(6):
        E.append(synth.Ellipse(rng.uniform(-0.2, 0.2) * g.nx * g.dx, rng.uniform(-0.2, 0.2) * g.ny * g.dy,
                               rng.uniform(0.03, 0.1) * g.nx * g.dx, rng.uniform(0.03, 0.1) * g.ny * g.dy,
                               rng.uniform(0, 3), rng.uniform(-0.005, 0.005)))
    x = synth.rasterize_ellipses(E, g.nx, g.ny, g.dx, g.dy, g.offset_x, g.offset_y, oversample=2)
    return x.astype(np.float32)


@pytest.mark.parametrize("gname", ["small", "fan2d_128"])
@pytest.mark.parametrize("kind", ["phantom", "random"])
def test_forward_parity(ct, make_geom, gname, kind):
    g = SMALL if gname == "small" else synth.fan2d_128().geom
    x = phantom_image(g) if kind == "phantom" else np.random.default_rng(1).random((g.ny, g.nx)).astype(np.float32)
    G = make_geom(g)
    y = torch.empty(g.na, g.ns, device="cuda")
    ct.ct_forward(G, dev(x), y)
    torch.cuda.synchronize()
    ref = FanProjector(g).forward(x.astype(np.float64))
    e = rel_err(y.cpu().numpy(), ref)
    print(f"forward {gname} {kind}: worst per-ray error {e:.2e}")
    assert e <= TOL_RAY


def test_forward_parity_fine_detector(ct):
    """Cells so narrow that one footprint covers up to 11 of them: the per-ray fallback kernel, at the
    same per-ray bound."""
    g = synth.FanArcGeometry(nx=40, ny=40, dx=1.0, dy=1.0, ns=300, ds=0.3, na=12, dso=300.0, dsd=500.0,
                             orbit_start_deg=3.0)
    x = phantom_image(g)
    G = ct.Geometry.from_fan(g)
    y = torch.empty(g.na, g.ns, device="cuda")
    ct.ct_forward(G, dev(x), y)
    torch.cuda.synchronize()
    ef = rel_err(y.cpu().numpy(), FanProjector(g).forward(x.astype(np.float64)))
    xb = torch.empty(g.ny, g.nx, device="cuda")
    ct.ct_back(G, y, xb)
    torch.cuda.synchronize()
    eb = rel_err(xb.cpu().numpy(), FanProjector(g).back(y.cpu().numpy().astype(np.float64)))
    print(f"fine detector: worst per-ray error {ef:.2e}, per-pixel {eb:.2e}")
    assert ef <= TOL_RAY and eb <= TOL_RAY


@pytest.mark.parametrize("gname", ["small", "fan2d_128"])
def test_back_parity(ct, make_geom, gname):
    g = SMALL if gname == "small" else synth.fan2d_128().geom
    P = FanProjector(g)
    G = make_geom(g)
    sino = P.forward(phantom_image(g).astype(np.float64)).astype(np.float32)  # positive sinogram
    x = torch.empty(g.ny, g.nx, device="cuda")
    ct.ct_back(G, dev(sino), x)
    torch.cuda.synchronize()
    ref = P.back(sino.astype(np.float64))
    e = rel_err(x.cpu().numpy(), ref)
    print(f"back {gname}: worst per-pixel error {e:.2e}")
    assert e <= TOL_RAY
    # signed data: error relative to the largest pixel
    r = np.random.default_rng(2).standard_normal((g.na, g.ns)).astype(np.float32)
    ct.ct_back(G, dev(r), x, scale=0.5)
    torch.cuda.synchronize()
    ref = 0.5 * P.back(r.astype(np.float64))
    assert np.max(np.abs(x.cpu().numpy() - ref)) <= 1e-5 * np.abs(ref).max()


def test_adjointness_gpu(ct, make_geom):
    g = synth.fan2d_128().geom
    G = make_geom(g)
    rng = np.random.default_rng(3)
    x = dev(rng.random((g.ny, g.nx)))
    yv = dev(rng.random((g.na, g.ns)))
    Ax = torch.empty(g.na, g.ns, device="cuda")
    Aty = torch.empty(g.ny, g.nx, device="cuda")
    ct.ct_forward(G, x, Ax)
    ct.ct_back(G, yv, Aty)
    a = float((Ax.double() * yv.double()).sum())
    b = float((x.double() * Aty.double()).sum())
    assert abs(a - b) <= 1e-5 * abs(a)


def test_view_lists_and_accumulate(ct, make_geom):
    g = SMALL
    P = FanProjector(g)
    G = make_geom(g)
    x = phantom_image(g)
    views = [44, 3, 17, 0, 29]
    y = torch.empty(len(views), g.ns, device="cuda")
    ct.ct_forward(G, dev(x), y, views=views)
    torch.cuda.synchronize()
    assert rel_err(y.cpu().numpy(), P.forward(x.astype(np.float64), views)) <= TOL_RAY
    base = np.random.default_rng(4).random((g.ny, g.nx)).astype(np.float32)
    xo = dev(base)
    ct.ct_back(G, y, xo, views=views, scale=2.0, accumulate=True)
    torch.cuda.synchronize()
    ref = base + 2.0 * P.back(y.cpu().numpy().astype(np.float64), views)
    assert rel_err(xo.cpu().numpy(), ref) <= TOL_RAY
    one = torch.empty(1, g.ns, device="cuda")
    ct.ct_forward(G, dev(x), one, views=[13])
    torch.cuda.synchronize()
    assert rel_err(one.cpu().numpy(), P.forward(x.astype(np.float64), [13])) <= TOL_RAY


def test_zero_image_and_bad_views(ct):
    g = SMALL
    G = ct.Geometry.from_fan(g)
    y = torch.full((g.na, g.ns), 7.0, device="cuda")
    ct.ct_forward(G, torch.zeros(g.ny, g.nx, device="cuda"), y)
    torch.cuda.synchronize()
    assert float(y.abs().max()) == 0.0
    with pytest.raises(ct.CTError) as e:
        ct.ct_forward(G, torch.zeros(g.ny, g.nx, device="cuda"), torch.empty(1, g.ns, device="cuda"), views=[g.na])
    assert e.value.status == ct.CT_EINVAL
    with pytest.raises(ct.CTError):
        ct.ct_forward(G, torch.zeros(g.ny, g.nx, device="cuda"), torch.empty(0, g.ns, device="cuda"), views=[])


def test_packed_image_and_forward(ct, make_geom):
    """ct_pack_image writes [x | x^T]; projecting the packed image gives ct_forward's rays exactly
    (with the resident matrix its steep rays read the transposed half)."""
    g = SMALL  # not square: nx != ny
    G = make_geom(g)
    x = dev(phantom_image(g))
    xp = torch.empty(2 * g.nx * g.ny, device="cuda")
    ct.ct_pack_image(G, x, xp)
    ref = torch.cat([x.reshape(-1), x.t().contiguous().reshape(-1)])
    assert torch.equal(xp, ref)
    y1 = torch.empty(g.na, g.ns, device="cuda")
    y2 = torch.empty_like(y1)
    ct.ct_forward(G, x, y1)
    ct.ct_forward_packed(G, xp, y2)
    assert torch.equal(y1, y2)
    views = [3, 44, 0, 21]
    y3 = torch.empty(len(views), g.ns, device="cuda")
    ct.ct_forward_packed(G, xp, y3, views=views)
    assert rel_err(y3.cpu().numpy(), y1[views].cpu().numpy()) <= 1e-6


def test_sqs_diag_parity(ct, make_geom):
    c = synth.fan2d_128()
    d = synth.make_scan(c)
    w = d.w.astype(np.float32)
    G = make_geom(c.geom)
    dl = torch.empty(c.geom.ny, c.geom.nx, device="cuda")
    ct.ct_sqs_diag(G, dev(w), dl)
    torch.cuda.synchronize()
    P = FanProjector(c.geom)
    ref = P.back(w.astype(np.float64) * P.forward(np.ones((c.geom.ny, c.geom.nx))))
    assert rel_err(dl.cpu().numpy(), ref) <= TOL_RAY


@pytest.mark.parametrize("pot", ["hyperbola", "fair", "quadratic"])
def test_reg_gradient_parity(ct, pot):
    g = SMALL
    G = ct.Geometry.from_fan(g)
    x = phantom_image(g) + 1e-4 * np.random.default_rng(5).standard_normal((g.ny, g.nx)).astype(np.float32)
    beta, delta = 3.0e6, 2e-4
    gr = torch.empty(g.ny, g.nx, device="cuda")
    cv = torch.empty(g.ny, g.nx, device="cuda")
    ct.ct_reg_gradient(G, dev(x), beta, delta, pot, gr, cv)
    torch.cuda.synchronize()
    x64 = x.astype(np.float64)
    rg = oreg.gradient(x64, beta, delta, pot)
    rc = oreg.curvature(x64, beta, delta, pot)
    assert np.max(np.abs(gr.cpu().numpy() - rg)) <= 1e-5 * np.abs(rg).max()
    assert rel_err(cv.cpu().numpy(), rc) <= 1e-5


def _solve_case(ct, c, M, alpha, n_iter, algorithm="proposed", continuation=True, rho_fixed=0.0, x0=None,
                make_geom=None, curvature="huber", dl_scale=1.0):
    d = synth.make_scan(c)
    y32, w32 = d.y.astype(np.float32), d.w.astype(np.float32)
    g = c.geom
    x0 = np.zeros((g.ny, g.nx), np.float32) if x0 is None else x0.astype(np.float32)
    prob = osolver.PWLSProblem(FanProjector(g), y32.astype(np.float64), w32.astype(np.float64),
                               c.beta_per_mm, c.delta, c.potential)
    xo = osolver.relaxed_os_lalm(prob, x0.astype(np.float64), M, alpha, n_iter, algorithm=algorithm,
                                 continuation=continuation, rho_fixed=rho_fixed, curvature=curvature,
                                 dl_scale=dl_scale)
    G = make_geom(g) if make_geom else ct.Geometry.from_fan(g)
    xg = dev(x0)
    ct.ct_relaxed_oslalm_solve(G, dev(y32), dev(w32), xg, M=M, n_iter=n_iter, alpha=alpha, beta=c.beta_per_mm,
                               delta=c.delta, potential=c.potential, algorithm=algorithm,
                               continuation=continuation, rho_fixed=rho_fixed, curvature=curvature, dl_scale=dl_scale)
    mask = osolver.fov_mask(g)
    return osolver.rmsd_hu(xg.cpu().numpy().astype(np.float64), xo, mask, c.hu_per_unit), xo


@pytest.mark.parametrize("M,alpha,n_iter,alg", [
    (10, 1.999, 20, "proposed"),   # the 128x128 workload as specified
    (5, 1.999, 20, "proposed"),
    (10, 1.0, 20, "proposed"),
    (10, 1.999, 10, "simple"),
    (1, 1.999, 15, "proposed"),
    (7, 1.5, 6, "proposed"),       # uneven subsets (180 = 7 * 25 + 5)
])
def test_solve_parity_fan2d_128(ct, make_geom, M, alpha, n_iter, alg):
    rmsd, _ = _solve_case(ct, synth.fan2d_128(), M, alpha, n_iter, algorithm=alg, make_geom=make_geom)
    assert rmsd <= 0.1, rmsd


@pytest.mark.parametrize("curvature,dl_scale", [("max", 1.0), ("huber", 2.0), ("max", 0.75)])
def test_solve_parity_majorizer_variants(ct, curvature, dl_scale):
    """The supplement's majorizer study: maximum-curvature D_R and scaled D_L, against the oracle."""
    rmsd, _ = _solve_case(ct, synth.fan2d_128(), 5, 1.999, 10, curvature=curvature, dl_scale=dl_scale)
    assert rmsd <= 0.1, rmsd


def test_solve_parity_fixed_rho(ct):
    # rho = 0.5 throughout (no continuation).  A rho as small as 0.05 from a zero
    # image overshoots to ~1000 HU in the first iteration, where FP32 and FP64
    # clip different pixels and the trajectories part; that is not a parity case.
    rmsd, _ = _solve_case(ct, synth.fan2d_128(), 5, 1.999, 8, continuation=False, rho_fixed=0.5)
    assert rmsd <= 0.1, rmsd


def test_solve_report_and_trace(ct):
    c = synth.fan2d_128()
    d = synth.make_scan(c)
    g = c.geom
    G = ct.Geometry.from_fan(g)
    y, w = dev(d.y), dev(d.w)
    xref = torch.zeros(g.ny, g.nx, device="cuda")
    ct.ct_relaxed_oslalm_solve(G, y, w, xref, M=1, n_iter=40, alpha=1.999, beta=c.beta_per_mm, delta=c.delta)
    x = torch.zeros(g.ny, g.nx, device="cuda")
    rep = ct.ct_relaxed_oslalm_solve(G, y, w, x, M=5, n_iter=6, alpha=1.999, beta=c.beta_per_mm, delta=c.delta,
                                     x_ref=xref, hu_per_unit=c.hu_per_unit)
    assert rep["iters_done"] == 6 and len(rep["rmsd_trace_hu"]) == 6
    mask = osolver.fov_mask(g)
    direct = osolver.rmsd_hu(x.cpu().numpy().astype(np.float64), xref.cpu().numpy().astype(np.float64), mask,
                             c.hu_per_unit)
    assert abs(rep["rmsd_trace_hu"][-1] - direct) <= 1e-4 * max(direct, 1.0)
    assert all(b >= a for a, b in zip(rep["iter_seconds"], rep["iter_seconds"][1:]))
    # early stop at a loose tolerance
    x2 = torch.zeros(g.ny, g.nx, device="cuda")
    tol = rep["rmsd_trace_hu"][2] + 1e-3
    rep2 = ct.ct_relaxed_oslalm_solve(G, y, w, x2, M=5, n_iter=6, alpha=1.999, beta=c.beta_per_mm, delta=c.delta,
                                      x_ref=xref, hu_per_unit=c.hu_per_unit, stop_rmsd_hu=tol)
    assert rep2["iters_done"] <= 3 and rep2["seconds_to_tol"] > 0


def test_full_size_sampled_parity(ct, make_geom):
    """512x512, 984 views x 888 bins (the clinical-scale workload): sampled rays and pixels."""
    c = synth.fan2d_512()
    g = c.geom
    d = synth.make_scan(c)
    x = synth.rasterize_ellipses(d.ellipses, g.nx, g.ny, g.dx, g.dy, oversample=2).astype(np.float32)
    G = make_geom(g)
    y = torch.empty(g.na, g.ns, device="cuda")
    ct.ct_forward(G, dev(x), y)
    yb = y.cpu().numpy()
    rng = np.random.default_rng(6)
    rv = rng.integers(0, g.na, 48)
    rb = rng.integers(0, g.ns, 48)
    P = FanProjector(g)
    ref = P.forward_rays(x.astype(np.float64), rv, rb)
    scale = np.abs(yb).max()
    den = np.maximum(np.abs(ref), 1e-3 * scale)
    assert np.max(np.abs(yb[rv, rb] - ref) / den) <= TOL_RAY
    # back-projection of the weighted residual-like sinogram at sampled pixels (a 41-subset's views)
    views = list(range(7, g.na, 41))
    sino = (d.w[views] * 1e-5).astype(np.float32)
    xb = torch.empty(g.ny, g.nx, device="cuda")
    ct.ct_back(G, dev(sino), xb, views=views)
    pix = rng.integers(0, g.nx * g.ny, 48)
    refp = P.back_pixels(sino.astype(np.float64), views, pix)
    got = xb.cpu().numpy().reshape(-1)[pix]
    den = np.maximum(np.abs(refp), 1e-3 * np.abs(xb.cpu().numpy()).max())
    assert np.max(np.abs(got - refp) / den) <= TOL_RAY


def test_resident_matrix_limit_and_size(ct):
    g = SMALL
    G = ct.Geometry.from_fan(g)
    with pytest.raises(ct.CTError) as e:
        ct.ct_geom_precompute(G, max_bytes=1024)
    assert e.value.status == ct.CT_ENOMEM
    # still usable on the fly after the refusal
    y = torch.empty(g.na, g.ns, device="cuda")
    ct.ct_forward(G, dev(phantom_image(g)), y)
    b = ct.ct_geom_precompute(G)
    ntiles = ((g.nx + 15) // 16) * ((g.ny + 15) // 16)
    # the records: per view and 32 pixels at least the 16-bit first cells and counts, two weights, a word
    m, r = ct.ct_geom_matrix_info(G)
    assert m == b and g.na * ntiles * 8 * (64 + 256 + 4) <= r < b
    assert ct.ct_geom_precompute(G) == b  # idempotent
    y2 = torch.empty_like(y)
    ct.ct_forward(G, dev(phantom_image(g)), y2)
    torch.cuda.synchronize()
    assert rel_err(y2.cpu().numpy(), y.cpu().numpy()) <= 2e-6
