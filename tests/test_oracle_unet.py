"""Pins of the FP64 U-Net reference (test infrastructure) against things other than itself:
* BF16 rounding against torch's bfloat16 conversion (round to nearest even);
* conv3x3 against scipy.signal.correlate2d summed over channel pairs;
* conv3x3_input_grad and conv3x3_weight_grad are the adjoints of conv3x3 in its input and
  weights; max-pool routing and nearest upsampling against their adjoint identities;
* the whole network's backward (FP64 mode) against central finite differences of its forward.
"""

import numpy as np
import pytest
import torch
from scipy.signal import correlate2d

from oracle import unet as ou


def test_bf16_round_matches_torch():
    x = np.random.default_rng(0).standard_normal(10000).astype(np.float32) * np.float32(3.7)
    x = np.concatenate([x, np.float32([1.0, 1.00390625, 1.0078125 * 1.001, 0.0, -2.5e-3])])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(ou.bf16_round(x), ref)


def test_conv3x3_matches_scipy():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 7, 9, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    out = ou.conv3x3(x, w)
    for b in range(2):
        for o in range(4):
            ref = sum(correlate2d(x[b, :, :, c], w[o, :, :, c], mode="same") for c in range(3))
            np.testing.assert_allclose(out[b, :, :, o], ref, rtol=1e-12, atol=1e-12)


def test_conv_adjoints():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 6, 5, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    g = rng.standard_normal((2, 6, 5, 4))
    lhs = np.sum(ou.conv3x3(x, w) * g)
    assert abs(lhs - np.sum(x * ou.conv3x3_input_grad(g, w))) <= 1e-12 * abs(lhs)
    assert abs(lhs - np.sum(w * ou.conv3x3_weight_grad(x, g))) <= 1e-12 * abs(lhs)


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 8, 6, 3))
    p, arg = ou.maxpool(x)
    gp = rng.standard_normal(p.shape)
    g = ou.maxpool_grad(gp, arg, x.shape)
    # the routed gradient is the derivative of sum(gp * maxpool(x)): finite difference on one element
    i = np.unravel_index(np.argmax(np.abs(g)), g.shape)
    e = np.zeros_like(x)
    e[i] = 1e-6
    fd = (np.sum(gp * ou.maxpool(x + e)[0]) - np.sum(gp * ou.maxpool(x - e)[0])) / 2e-6
    assert abs(fd - g[i]) < 1e-6
    u = rng.standard_normal((2, 4, 3, 3))
    gu = rng.standard_normal((2, 8, 6, 3))
    assert abs(np.sum(ou.upsample(u) * gu) - np.sum(u * ou.upsample_grad(gu))) < 1e-10


def _random_net(levels=3, base=16, seed=0):
    rng = np.random.default_rng(seed)
    probe = ou.UNetRef(levels, base, 2.0, np.zeros(_count(levels, base)))
    p = np.zeros(probe.nparams)
    for name, (o, ob, ci, co) in probe.offsets.items():
        p[o:ob] = rng.standard_normal(ob - o) * np.sqrt(2.0 / (9 * ci))
        p[ob:ob + co] = rng.standard_normal(co) * 0.05
    p[probe.out_off:] = rng.standard_normal(base + 1) * 0.1
    return ou.UNetRef(levels, base, 2.0, p)


def _count(levels, base):
    ch = [base << l for l in range(levels)]
    n = 0
    for l in range(levels):
        ci = 1 if l == 0 else ch[l - 1]
        n += ch[l] * 9 * ci + ch[l] + ch[l] * 9 * ch[l] + ch[l]
    for l in range(levels - 2, -1, -1):
        n += ch[l] * 9 * (ch[l + 1] + ch[l]) + ch[l] + ch[l] * 9 * ch[l] + ch[l]
    return n + base + 1


def test_network_backward_matches_finite_differences():
    net = _random_net()
    rng = np.random.default_rng(5)
    x = rng.random((2, 16, 16)) + 0.2
    gy = rng.standard_normal((2, 16, 16))
    _, cache = net.forward(x, bf16=False)
    g = net.pack(net.backward(gy, cache, bf16=False))
    f = lambda p: np.sum(gy * ou.UNetRef(3, 16, 2.0, p).forward(x, bf16=False)[0])  # noqa: E731
    picks = []
    for name, (o, ob, ci, co) in list(net.offsets.items()):
        picks += [o + int(rng.integers(0, ob - o)), ob + int(rng.integers(0, co))]
    picks += [net.out_off + 3, net.out_off + net.C0]
    eps = 1e-5
    for i in picks:
        pp, pm = net.p.copy(), net.p.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (f(pp) - f(pm)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(g[i])) + 1e-7, (i, fd, g[i])
