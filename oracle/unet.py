"""FP64 reference of the warm-start U-Net: forward and backward, written out layer by layer.

ORACLE -- test infrastructure only.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this module.

The network (architecture, parameter layout) is the one documented in
include/ct_unet.h.  Every sum is taken in FP64.  With ``bf16=True`` the
reference rounds the tensors the GPU stores in BF16 (inputs of each
convolution, weights, activations and activation gradients) at the same
points (round to nearest even), so that a comparison with the GPU measures
only its FP32 accumulation order; with ``bf16=False`` it is the plain FP64
network, used for the finite-difference pins of its backward pass.
"""

from __future__ import annotations

import numpy as np


def bf16_round(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), via the FP32 bit pattern; returns float64."""
    a32 = np.ascontiguousarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3x3(x: np.ndarray, w: np.ndarray) -> np.ndarray:
    """out[b, y, x, o] = sum_{ky, kx, c} w[o, ky, kx, c] x[b, y + ky - 1, x + kx - 1, c] (zero padding)."""
    B, H, W, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    out = np.zeros((B, H, W, w.shape[0]))
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("bhwc,oc->bhwo", xp[:, ky:ky + H, kx:kx + W, :], w[:, ky, kx, :])
    return out


def conv3x3_input_grad(g: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Adjoint of conv3x3 in its input: gx[b, y, x, c] = sum g[b, y - ky + 1, x - kx + 1, o] w[o, ky, kx, c]."""
    B, H, W, _ = g.shape
    gp = np.pad(g, ((0, 0), (1, 1), (1, 1), (0, 0)))
    out = np.zeros((B, H, W, w.shape[3]))
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("bhwo,oc->bhwc", gp[:, 2 - ky:2 - ky + H, 2 - kx:2 - kx + W, :], w[:, ky, kx, :])
    return out


def conv3x3_weight_grad(x: np.ndarray, g: np.ndarray) -> np.ndarray:
    """dw[o, ky, kx, c] = sum_{b, y, x} g[b, y, x, o] x[b, y + ky - 1, x + kx - 1, c]."""
    B, H, W, C = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dw = np.zeros((g.shape[3], 3, 3, C))
    for ky in range(3):
        for kx in range(3):
            dw[:, ky, kx, :] = np.einsum("bhwo,bhwc->oc", g, xp[:, ky:ky + H, kx:kx + W, :])
    return dw


def maxpool(x: np.ndarray):
    """2x2 max pooling; also returns, per output element, the index (0..3, order (0,0),(0,1),(1,0),(1,1))
    of the first maximal input."""
    B, H, W, C = x.shape
    v = np.stack([x[:, 0::2, 0::2], x[:, 0::2, 1::2], x[:, 1::2, 0::2], x[:, 1::2, 1::2]], axis=0)
    arg = np.argmax(v, axis=0)  # first maximum
    return np.max(v, axis=0), arg


def maxpool_grad(gp: np.ndarray, arg: np.ndarray, shape) -> np.ndarray:
    g = np.zeros(shape)
    for k, (dy, dx) in enumerate(((0, 0), (0, 1), (1, 0), (1, 1))):
        g[:, dy::2, dx::2] = np.where(arg == k, gp, 0.0)
    return g


def upsample(x: np.ndarray) -> np.ndarray:
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample_grad(g: np.ndarray) -> np.ndarray:
    return g[:, 0::2, 0::2] + g[:, 0::2, 1::2] + g[:, 1::2, 0::2] + g[:, 1::2, 1::2]


class UNetRef:
    """The U-Net of include/ct_unet.h with its parameters unpacked from the flat FP32 vector."""

    def __init__(self, levels: int, base: int, in_scale: float, params: np.ndarray):
        self.L, self.C0, self.s = levels, base, float(in_scale)
        ch = [base << l for l in range(levels)]
        self.layers = []  # (name, c_in, c_out)
        for l in range(levels):
            self.layers.append((f"enc{l}a", 1 if l == 0 else ch[l - 1], ch[l]))
            self.layers.append((f"enc{l}b", ch[l], ch[l]))
        for l in range(levels - 2, -1, -1):
            self.layers.append((f"dec{l}a", ch[l + 1] + ch[l], ch[l]))
            self.layers.append((f"dec{l}b", ch[l], ch[l]))
        self.ch = ch
        self.offsets = {}
        off = 0
        for name, ci, co in self.layers:
            self.offsets[name] = (off, off + co * 9 * ci, ci, co)
            off += co * 9 * ci + co
        self.out_off = off
        self.nparams = off + base + 1
        p = np.asarray(params, dtype=np.float64)
        assert p.size == self.nparams, (p.size, self.nparams)
        self.p = p

    def W(self, name):
        o, ob, ci, co = self.offsets[name]
        return self.p[o:ob].reshape(co, 3, 3, ci), self.p[ob:ob + co]

    def pack(self, grads: dict) -> np.ndarray:
        out = np.zeros(self.nparams)
        for name, (o, ob, ci, co) in self.offsets.items():
            out[o:ob] = grads[name][0].reshape(-1)
            out[ob:ob + co] = grads[name][1]
        out[self.out_off:self.out_off + self.C0] = grads["out"][0]
        out[self.out_off + self.C0] = grads["out"][1]
        return out

    def forward(self, x: np.ndarray, bf16: bool = True):
        """x [B][H][W] -> y [B][H][W]; returns (y, cache)."""
        r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))  # noqa: E731
        L = self.L
        c = {"x": np.asarray(x, dtype=np.float64)}
        xs = r(np.float32(self.s) * np.asarray(x, dtype=np.float32)) if bf16 else self.s * c["x"]
        c["xs"] = xs[..., None]
        w, b = self.W("enc0a")
        a = [None] * L
        s = [None] * L
        p = [None] * L
        parg = [None] * L
        a[0] = r(np.maximum(conv3x3(c["xs"], r(w)) + b, 0.0))
        for l in range(L):
            if l > 0:
                p[l - 1], parg[l - 1] = maxpool(s[l - 1])
                w, b = self.W(f"enc{l}a")
                a[l] = r(np.maximum(conv3x3(p[l - 1], r(w)) + b, 0.0))
            w, b = self.W(f"enc{l}b")
            s[l] = r(np.maximum(conv3x3(a[l], r(w)) + b, 0.0))
        e = [None] * L
        f = [None] * L
        T = s[L - 1]
        for l in range(L - 2, -1, -1):
            w, b = self.W(f"dec{l}a")
            cat = np.concatenate([upsample(T), s[l]], axis=3)
            e[l] = r(np.maximum(conv3x3(cat, r(w)) + b, 0.0))
            w, b = self.W(f"dec{l}b")
            f[l] = r(np.maximum(conv3x3(e[l], r(w)) + b, 0.0))
            T = f[l]
        wo = self.p[self.out_off:self.out_off + self.C0]
        bo = self.p[self.out_off + self.C0]
        y = c["x"] + (bo + np.einsum("bhwc,c->bhw", f[0], r(wo))) / self.s
        c.update(a=a, s=s, p=p, parg=parg, e=e, f=f)
        return y, c

    def backward(self, gy: np.ndarray, c: dict, bf16: bool = True) -> dict:
        """Parameter gradients of sum(gy * y) for the forward that produced cache c."""
        r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))  # noqa: E731
        L = self.L
        a, s, p, parg, e, f = c["a"], c["s"], c["p"], c["parg"], c["e"], c["f"]
        grads = {}
        gz = np.asarray(gy, dtype=np.float64) / self.s
        wo = self.p[self.out_off:self.out_off + self.C0]
        grads["out"] = (np.einsum("bhw,bhwc->c", gz, f[0]), gz.sum())
        g = r(gz[..., None] * r(wo) * (f[0] > 0))
        gs = [None] * L
        for l in range(0, L - 1):
            w, _ = self.W(f"dec{l}b")
            grads[f"dec{l}b"] = (conv3x3_weight_grad(e[l], g), g.sum(axis=(0, 1, 2)))
            ge = r(conv3x3_input_grad(g, r(w)) * (e[l] > 0))
            T = s[L - 1] if l + 1 == L - 1 else f[l + 1]
            cat = np.concatenate([upsample(T), s[l]], axis=3)
            w, _ = self.W(f"dec{l}a")
            grads[f"dec{l}a"] = (conv3x3_weight_grad(cat, ge), ge.sum(axis=(0, 1, 2)))
            gcat = conv3x3_input_grad(ge, r(w)) * (cat > 0)
            cu = self.ch[l + 1]
            gup = r(gcat[..., :cu])
            gs[l] = r(gcat[..., cu:])
            g = r(upsample_grad(gup))
        for l in range(L - 1, -1, -1):
            gsl = g if l == L - 1 else gs[l]
            w, _ = self.W(f"enc{l}b")
            grads[f"enc{l}b"] = (conv3x3_weight_grad(a[l], gsl), gsl.sum(axis=(0, 1, 2)))
            ga = r(conv3x3_input_grad(gsl, r(w)) * (a[l] > 0))
            if l == 0:
                grads["enc0a"] = (conv3x3_weight_grad(c["xs"], ga), ga.sum(axis=(0, 1, 2)))
            else:
                w, _ = self.W(f"enc{l}a")
                grads[f"enc{l}a"] = (conv3x3_weight_grad(p[l - 1], ga), ga.sum(axis=(0, 1, 2)))
                gp = r(conv3x3_input_grad(ga, r(w)) * (p[l - 1] > 0))
                routed = maxpool_grad(gp, parg[l - 1], s[l - 1].shape)
                gs[l - 1] = r(gs[l - 1] + routed)
        return grads
