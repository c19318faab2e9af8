"""The allocation-free D_L entry point against ct_sqs_diag, on consecutive calls.

ct_sqs_diag_noalloc serves callers that cannot allocate device memory once
running (a pool-reserved serving process, a latency-critical loop that must
not enter cudaMalloc/cudaFree).  Its scratch is a fixed device array shared by
all calls, so two calls in a row with different weights must each match the
workspace-based entry point, and so must a call on a smaller geometry right
after one on a larger one (a stale tail of the larger sinogram, or a wrong row
stride, would show).  The file sorts last so that a run stopping at its first
failure has run every other GPU test first; no other test depends on the
array, and these tests pass alone in a fresh process as well.
"""

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

SMALL = synth.FanArcGeometry(nx=37, ny=21, dx=1.1, dy=0.9, ns=61, ds=1.3, na=45, dso=200.0, dsd=350.0,
                             offset_x=0.3, offset_y=-0.45, offset_s=0.25, orbit_start_deg=7.0, orbit_deg=300.0)


def _rel_err(got, ref):
    den = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    return float(np.max(np.abs(got - ref) / den))


@pytest.mark.parametrize("resident", [False, True])
@pytest.mark.parametrize("gname", ["small", "fan2d_128"])
def test_noalloc_matches_sqs_diag_on_consecutive_calls(gname, resident):
    from paper_1512_04564_gb300 import ct

    g = SMALL if gname == "small" else synth.fan2d_128().geom
    G = ct.Geometry.from_fan(g)
    if resident:
        ct.ct_geom_precompute(G)
    rng = np.random.default_rng(7)
    for call in range(2):
        w = torch.from_numpy((rng.random((g.na, g.ns)) * 1e4 + 1.0).astype(np.float32)).cuda()
        ref = torch.empty(g.ny, g.nx, device="cuda")
        ct.ct_sqs_diag(G, w, ref)
        out = torch.full((g.ny, g.nx), float("nan"), device="cuda")
        ct.ct_sqs_diag_noalloc(G, w, out)
        torch.cuda.synchronize()
        assert _rel_err(out.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)) <= 1e-5, call


@pytest.mark.parametrize("resident", [False, True])
def test_noalloc_larger_then_smaller_geometry(resident):
    from paper_1512_04564_gb300 import ct

    rng = np.random.default_rng(8)
    for g in (synth.fan2d_128().geom, SMALL):  # 180 x 256 cells, then 45 x 61 with a different row length
        G = ct.Geometry.from_fan(g)
        if resident:
            ct.ct_geom_precompute(G)
        w = torch.from_numpy((rng.random((g.na, g.ns)) * 1e4 + 1.0).astype(np.float32)).cuda()
        out = torch.full((g.ny, g.nx), float("nan"), device="cuda")
        ct.ct_sqs_diag_noalloc(G, w, out)  # before ct_sqs_diag: no ray sums kept yet (forward pass)
        ref = torch.empty(g.ny, g.nx, device="cuda")
        ct.ct_sqs_diag(G, w, ref)
        out2 = torch.full((g.ny, g.nx), float("nan"), device="cuda")
        ct.ct_sqs_diag_noalloc(G, w, out2)  # after it: from the kept ray sums
        torch.cuda.synchronize()
        r = ref.cpu().numpy().astype(np.float64)
        assert _rel_err(out.cpu().numpy().astype(np.float64), r) <= 1e-5
        assert _rel_err(out2.cpu().numpy().astype(np.float64), r) <= 1e-5


def test_noalloc_rejects_oversized_sinogram():
    from paper_1512_04564_gb300 import ct

    g = synth.FanArcGeometry(nx=64, ny=64, dx=1.0, dy=1.0, ns=1100, ds=0.5, na=1000, dso=541.0, dsd=949.0)
    G = ct.Geometry.from_fan(g)
    w = torch.ones(g.na, g.ns, device="cuda")
    d = torch.empty(g.ny, g.nx, device="cuda")
    with pytest.raises(ct.CTError) as e:
        ct.ct_sqs_diag_noalloc(G, w, d)
    assert e.value.status == ct.CT_EINVAL and "4 MiB" in str(e.value)
