"""Checkpoint and resume of relaxed OS-LALM (Algorithm 1 / 2 of Sec. III-A).

The solver state after outer iteration k is (x, g, h, k): D_L is recomputed
from the weights, rho depends only on the subiteration count (Eq. (dec_rho)),
and the next subset is the first.  A solve of n1 iterations that writes its
final g and h, resumed for n2 more iterations, must give the same x, g and h,
bit for bit, as one run of n1 + n2 iterations on the same GPU (the projectors
add in a fixed order, with no atomics on data).
"""

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _run(ct, G, y, w, shape, kw, n1, n2):
    xa = torch.zeros(shape, device="cuda")
    ga, ha = torch.empty(shape, device="cuda"), torch.empty(shape, device="cuda")
    ct.ct_relaxed_oslalm_solve(G, y, w, xa, n_iter=n1 + n2, g_state=ga, h_state=ha, **kw)
    xb = torch.zeros(shape, device="cuda")
    gb, hb = torch.empty(shape, device="cuda"), torch.empty(shape, device="cuda")
    ct.ct_relaxed_oslalm_solve(G, y, w, xb, n_iter=n1, g_state=gb, h_state=hb, **kw)
    kw2 = dict(kw, init_fbp=False)
    ct.ct_relaxed_oslalm_solve(G, y, w, xb, n_iter=n2, start_iter=n1, g_state=gb, h_state=hb, **kw2)
    torch.cuda.synchronize()
    return (xa, ga, ha), (xb, gb, hb)


@pytest.mark.parametrize("path,algorithm", [("on_the_fly", "proposed"), ("resident_matrix", "proposed"),
                                            ("resident_matrix", "simple")])
def test_resume_is_bit_identical_2d(path, algorithm):
    from paper_1512_04564_gb300 import ct

    c = synth.fan2d_128()
    g = c.geom
    d = synth.make_scan(c)
    G = ct.Geometry.from_fan(g)
    if path == "resident_matrix":
        ct.ct_geom_precompute(G)
    y = torch.from_numpy(d.y.astype(np.float32)).cuda()
    w = torch.from_numpy(d.w.astype(np.float32)).cuda()
    kw = dict(M=10, alpha=1.999, beta=c.beta_per_mm, delta=c.delta, algorithm=algorithm, init_fbp=True)
    a, b = _run(ct, G, y, w, (g.ny, g.nx), kw, 3, 4)
    for u, v, name in zip(a, b, ("x", "g", "h")):
        assert torch.equal(u, v), name
    # and the state moved: resuming from the wrong iteration count changes rho and the result
    xc = a[0].clone()
    gc, hc = a[1].clone(), a[2].clone()
    xw = torch.zeros_like(xc)
    gw, hw = torch.empty_like(gc), torch.empty_like(hc)
    ct.ct_relaxed_oslalm_solve(G, y, w, xw, n_iter=3, g_state=gw, h_state=hw, **kw)
    ct.ct_relaxed_oslalm_solve(G, y, w, xw, n_iter=4, start_iter=1, g_state=gw, h_state=hw,
                               **dict(kw, init_fbp=False))
    torch.cuda.synchronize()
    assert not torch.equal(xw, xc)


def test_resume_is_bit_identical_helical():
    from paper_1512_04564_gb300 import ct

    c = synth.helix3d_64()
    g = c.geom
    d = synth.make_scan(c)
    G = ct.Geometry.from_helix(g)
    y = torch.from_numpy(d.y.astype(np.float32)).cuda()
    w = torch.from_numpy(d.w.astype(np.float32)).cuda()
    kw = dict(M=8, alpha=1.999, beta=c.beta_per_mm, delta=c.delta, init_fbp=True)
    a, b = _run(ct, G, y, w, (g.nz, g.ny, g.nx), kw, 2, 2)
    for u, v, name in zip(a, b, ("x", "g", "h")):
        assert torch.equal(u, v), name


def test_resume_needs_the_state():
    from paper_1512_04564_gb300 import ct

    c = synth.fan2d_128()
    g = c.geom
    G = ct.Geometry.from_fan(g)
    z = torch.zeros(g.na, g.ns, device="cuda")
    x = torch.zeros(g.ny, g.nx, device="cuda")
    with pytest.raises(ct.CTError) as e:
        ct.ct_relaxed_oslalm_solve(G, z, z + 1.0, x, M=10, n_iter=1, alpha=1.999, beta=1.0, delta=1.0, start_iter=2)
    assert e.value.status == ct.CT_EINVAL
