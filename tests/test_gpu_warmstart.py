"""The learned warm start end to end on a small version of its workload: pairs generated by the
solver, training on the GPU with the tensor-core U-Net and the data-consistency term through the
differentiable projector, and the gain over the plain FBP start on held-out problems (fewer
relaxed OS-LALM iterations to 1 HU of x*, and a start closer to x* than the FBP image)."""

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

MU_W = 0.02


def test_warm_start_beats_fbp_start():
    from paper_1512_04564_gb300 import ct, warmstart

    g = synth.warmstart_geometry(128, pixel=1.96)  # 128x128 over 250 mm, 222 bins, 246 views
    n_train, n_eval = 64, 12
    y, w = synth.warmstart.problems(range(n_train + n_eval), g, n_gauss=1)
    G = ct.Geometry.from_fan(g)
    ct.ct_geom_precompute(G)
    ys, ws = torch.from_numpy(y).cuda(), torch.from_numpy(w).cuda()
    beta, delta = 2.0 ** 14 / MU_W ** 2, 10 * MU_W / 1000
    xstar = warmstart.solve_xstar(G, ys, ws, beta, delta, os_iters=20, m1_iters=150, M=5)
    fbp = warmstart.fbp_images(G, ys)
    net = ct.UNet(levels=4, base_channels=16, height=128, width=128, max_batch=8, in_scale=1 / MU_W, seed=1)
    hist = warmstart.train(net, G, fbp[:n_train], xstar[:n_train], ys[:n_train], ws[:n_train], epochs=25, batch=8,
                           lr=2e-3, lr_min=1e-4, lam_dc=1e-4)
    assert hist[-1] < 0.5 * hist[0], hist
    res = warmstart.evaluate(net, G, ys[n_train:], ws[n_train:], xstar[n_train:], beta=beta, delta=delta, M=5,
                             n_iter=40)
    assert res["plain_iters"]["reached"] == n_eval and res["warm_iters"]["reached"] == n_eval, res
    assert res["warm_start_rmsd_hu"]["mean"] < 0.7 * res["fbp_rmsd_hu"]["mean"], res
    assert res["warm_iters"]["mean"] < res["plain_iters"]["mean"], res
