"""Plain FP64 CPU oracle of the learned seismogram surrogate (MLP + 1D-convolution decoder).

TEST INFRASTRUCTURE ONLY. The product (the CUDA library and its binding) never imports,
links or runs this file; only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU legs do. It shares no code with the CUDA path: every layer is written here from its
definition with numpy in float64.

The surrogate is not in the paper: it maps a source (location and moment tensor, 9 inputs)
to the three-component traces of the surface receivers for one fixed medium, trained on
runs of the spectral-element solver of Sec. II-B / V-C. Network (sizes from the caller):

    h1 = gelu(x W1^T + b1)                  9   -> 512
    h2 = gelu(h1 W2^T + b2)                 512 -> 512
    z  = gelu(h2 W3^T + b3), as [C0, L0]    512 -> C0 * L0
    for each decoder stage s: z = act_s(conv3(up_s(z)) + c_s)
    y  = z                                  [C_out = 3 * nrec, L]
    or, with a moment contraction of the last K inputs (z then has K * C_out channels),
    y[c, t] = sum_k x[9 - K + k] z[k * C_out + c, t]

with up_s = nearest-neighbour upsampling by 1 or 2 along time, conv3 a 'same' convolution
of width 3 (zero padding 1) over all input channels, act_s = gelu except the last stage
(identity). gelu is the tanh form 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))).
The loss is the mean squared error over all outputs.

Parity status: pinned by tests/test_oracle_surrogate.py (finite differences of the loss
for every parameter tensor, the convolution against numpy.convolve, gelu closed forms).
"""
from __future__ import annotations

import numpy as np

GELU_C = np.sqrt(2.0 / np.pi)
GELU_A = 0.044715


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(GELU_C * (x + GELU_A * x ** 3)))


def gelu_grad(x):
    """d gelu / dx of the tanh form."""
    u = GELU_C * (x + GELU_A * x ** 3)
    t = np.tanh(u)
    du = GELU_C * (1.0 + 3.0 * GELU_A * x ** 2)
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * du


def upsample(x, factor: int):
    """Nearest-neighbour upsampling along the last axis: y[..., t] = x[..., t // factor]."""
    return np.repeat(x, factor, axis=-1) if factor > 1 else x


def upsample_backward(dy, factor: int):
    if factor == 1:
        return dy
    shape = dy.shape[:-1] + (dy.shape[-1] // factor, factor)
    return dy.reshape(shape).sum(axis=-1)


def conv3(x, w, b):
    """'Same' width-3 convolution (cross-correlation, as in deep-learning frameworks):
    y[n, o, t] = b[o] + sum_{c, d} w[o, c, d] x[n, c, t + d - 1], x zero outside [0, L)."""
    L = x.shape[-1]
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1)))
    y = np.broadcast_to(b[None, :, None], (x.shape[0], w.shape[0], L)).copy()
    for d in range(3):
        y += np.einsum("oc,nct->not", w[:, :, d], xp[:, :, d:d + L])
    return y


def conv3_backward(x, w, dy):
    """Gradients of conv3 with respect to x, w and b."""
    L = x.shape[-1]
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1)))
    dw = np.stack([np.einsum("not,nct->oc", dy, xp[:, :, d:d + L]) for d in range(3)], axis=-1)
    db = dy.sum(axis=(0, 2))
    dxp = np.zeros_like(xp)
    for d in range(3):
        dxp[:, :, d:d + L] += np.einsum("oc,not->nct", w[:, :, d], dy)
    return dxp[:, :, 1:L + 1], dw, db


class Surrogate:
    """Parameters as float64 arrays (the CUDA side keeps bfloat16 copies of the weights;
    tests pass the same bf16-rounded values here)."""

    def __init__(self, params: dict, c0: int, l0: int, stages, contract: int = 0, bf16_operands: bool = False):
        """``stages``: list of (c_in, c_out, up) for the decoder; params holds W1, b1, W2, b2,
        W3, b3 and C{s}, c{s} (conv weight [c_out, c_in, 3], bias [c_out]) per stage. With
        ``contract`` = K > 0 the last stage's K * C channels D combine with the last K inputs:
        y[n, c, t] = sum_k x[n, -K + k] D[n, k * C + c, t] (seismograms are linear in the
        moment tensor)."""
        self.p = {k: np.asarray(v, dtype=np.float64) for k, v in params.items()}
        self.c0, self.l0 = c0, l0
        self.stages = list(stages)
        self.contract = int(contract)
        # with bf16_operands every operand of a weight product (activations, gradients) is
        # rounded to bfloat16 first, as on tensor cores; sums, biases, activations and the
        # moment contraction stay exact
        self.q = bf16_round if bf16_operands else (lambda v: v)

    def _combine(self, x, D):
        K = self.contract
        n, KC, L = D.shape
        return np.einsum("nk,nkct->nct", x[:, x.shape[1] - K:], D.reshape(n, K, KC // K, L))

    def _combine_backward(self, x, dy):
        K = self.contract
        return np.einsum("nk,nct->nkct", x[:, x.shape[1] - K:], dy).reshape(dy.shape[0], -1, dy.shape[2])

    def forward(self, x):
        """Returns (y [n, C_out, L], cache)."""
        p, q = self.p, self.q
        cache = {"x": x}
        a1 = q(x) @ p["W1"].T + p["b1"]
        h1 = gelu(a1)
        a2 = q(h1) @ p["W2"].T + p["b2"]
        h2 = gelu(a2)
        a3 = q(h2) @ p["W3"].T + p["b3"]
        z = gelu(a3).reshape(x.shape[0], self.c0, self.l0)
        cache.update(a1=a1, h1=h1, a2=a2, h2=h2, a3=a3)
        last = len(self.stages) - 1
        for s, (_, _, up) in enumerate(self.stages):
            zi = upsample(z, up)
            pre = conv3(q(zi), p[f"C{s}"], p[f"c{s}"])
            cache[f"in{s}"] = zi
            cache[f"pre{s}"] = pre
            z = pre if s == last else gelu(pre)
        if self.contract:
            z = self._combine(x, z)
        return z, cache

    def loss(self, x, target):
        y, _ = self.forward(x)
        return float(np.mean((y - target) ** 2))

    def backward(self, x, target):
        """Loss and its gradient for every parameter (dict of arrays)."""
        p, q = self.p, self.q
        y, c = self.forward(x)
        n_out = y.size
        g = {}
        dz = 2.0 * (y - target) / n_out
        if self.contract:
            dz = self._combine_backward(x, dz)
        last = len(self.stages) - 1
        for s in range(last, -1, -1):
            up = self.stages[s][2]
            dpre = dz if s == last else dz * gelu_grad(c[f"pre{s}"])
            dzi, g[f"C{s}"], _ = conv3_backward(q(c[f"in{s}"]), p[f"C{s}"], q(dpre))
            g[f"c{s}"] = dpre.sum(axis=(0, 2))
            dz = upsample_backward(dzi, up)
        da3 = dz.reshape(x.shape[0], -1) * gelu_grad(c["a3"])
        g["W3"] = q(da3).T @ q(c["h2"])
        g["b3"] = da3.sum(axis=0)
        da2 = (q(da3) @ p["W3"]) * gelu_grad(c["a2"])
        g["W2"] = q(da2).T @ q(c["h1"])
        g["b2"] = da2.sum(axis=0)
        da1 = (q(da2) @ p["W2"]) * gelu_grad(c["a1"])
        g["W1"] = q(da1).T @ q(x)
        g["b1"] = da1.sum(axis=0)
        return float(np.mean((y - target) ** 2)), g


def adam_step(param, grad, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (Kingma and Ba, ICLR 2015) in place; returns nothing."""
    m *= beta1
    m += (1.0 - beta1) * grad
    v *= beta2
    v += (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    param -= lr * mhat / (np.sqrt(vhat) + eps)


def bf16_round(x):
    """Round float64 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> np.uint64(16)) & np.uint64(1)
    rounded = ((bits + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)
