"""Pins of the surrogate network oracle: every layer against a definition written another
way (explicit loops, numpy.convolve, closed forms, adjoint identities), the full network's
gradients against central finite differences of the loss (FP64), Adam's first step and the
bfloat16 rounding against exact values."""
import numpy as np
import pytest

from paper_2606_12850_gb300 import inputs


@pytest.fixture(scope="module")
def so():
    from oracle import surrogate_oracle
    return surrogate_oracle


def tiny_net(so, seed=3):
    stages = [(4, 5, 2), (5, 5, 2), (5, 3, 1)]
    sizes = {"W1": (6, 9), "b1": (6,), "W2": (6, 6), "b2": (6,), "W3": (4 * 5, 6), "b3": (20,)}
    for s, (ci, co, _) in enumerate(stages):
        sizes[f"C{s}"] = (co, ci, 3)
        sizes[f"c{s}"] = (co,)
    params = {k: inputs.uniform(seed, v, -0.6, 0.6, stream=i) for i, (k, v) in enumerate(sizes.items())}
    return so.Surrogate(params, 4, 5, stages)


def test_gelu_closed_forms(so):
    x = np.linspace(-6, 6, 101)
    assert so.gelu(0.0) == 0.0
    np.testing.assert_allclose(so.gelu(x) - so.gelu(-x), x, rtol=0, atol=1e-14)  # tanh is odd
    assert abs(so.gelu(40.0) - 40.0) < 1e-12 and abs(so.gelu(-40.0)) < 1e-12
    h = 1e-6
    fd = (so.gelu(x + h) - so.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(so.gelu_grad(x), fd, rtol=0, atol=1e-8)


def test_conv3_against_loops_and_numpy(so):
    x = inputs.uniform(1, (2, 3, 11), -1, 1)
    w = inputs.uniform(2, (4, 3, 3), -1, 1)
    b = inputs.uniform(3, (4,), -1, 1)
    y = so.conv3(x, w, b)
    ref = np.zeros_like(y)
    for n in range(2):
        for o in range(4):
            for t in range(11):
                acc = b[o]
                for c in range(3):
                    for d in range(3):
                        s = t + d - 1
                        if 0 <= s < 11:
                            acc += w[o, c, d] * x[n, c, s]
                ref[n, o, t] = acc
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-13)
    # one channel: cross-correlation = convolution with the reversed kernel
    y1 = so.conv3(x[:1, :1], w[:1, :1], np.zeros(1))[0, 0]
    np.testing.assert_allclose(y1, np.convolve(x[0, 0], w[0, 0, ::-1], mode="same"), rtol=0, atol=1e-13)


def test_conv3_backward_is_the_adjoint(so):
    x = inputs.uniform(4, (2, 3, 9), -1, 1)
    w = inputs.uniform(5, (4, 3, 3), -1, 1)
    dy = inputs.uniform(6, (2, 4, 9), -1, 1)
    dx, dw, db = so.conv3_backward(x, w, dy)
    # <conv(x), dy> is bilinear: its derivative in x along x2 is <conv_nobias(x2), dy>
    x2 = inputs.uniform(7, x.shape, -1, 1)
    w2 = inputs.uniform(8, w.shape, -1, 1)
    zero = np.zeros(4)
    assert abs(np.sum(so.conv3(x2, w, zero) * dy) - np.sum(dx * x2)) < 1e-12
    assert abs(np.sum(so.conv3(x, w2, zero) * dy) - np.sum(dw * w2)) < 1e-12
    np.testing.assert_allclose(db, dy.sum(axis=(0, 2)), rtol=0, atol=1e-14)


def test_upsample_adjoint(so):
    x = inputs.uniform(9, (2, 3, 5), -1, 1)
    y = inputs.uniform(10, (2, 3, 10), -1, 1)
    assert abs(np.sum(so.upsample(x, 2) * y) - np.sum(x * so.upsample_backward(y, 2))) < 1e-13
    assert np.array_equal(so.upsample(x, 2)[..., 1::2], x)


def test_network_gradients_match_finite_differences(so):
    net = tiny_net(so)
    x = inputs.uniform(11, (3, 9), -1, 1)
    target = inputs.uniform(12, (3, 3, 20), -1, 1)
    _, grads = net.backward(x, target)
    for k in net.p:
        d = inputs.uniform(13, net.p[k].shape, -1, 1, stream=len(k))
        h = 1e-5
        base = net.p[k].copy()
        net.p[k] = base + h * d
        lp = net.loss(x, target)
        net.p[k] = base - h * d
        lm = net.loss(x, target)
        net.p[k] = base
        fd = (lp - lm) / (2 * h)
        an = float(np.sum(grads[k] * d))
        assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-12), (k, fd, an)


@pytest.mark.parametrize("mutation", ["gelu_grad", "conv_flip", "upsample_back"])
def test_planted_network_mistake_is_caught(so, monkeypatch, mutation):
    """A wrong activation derivative, a flipped convolution tap in the backward pass or a
    dropped upsampling sum each break the finite-difference pin."""
    if mutation == "gelu_grad":
        monkeypatch.setattr(so, "gelu_grad", lambda x: 0.5 * (1.0 + np.tanh(so.GELU_C * x)))
    elif mutation == "conv_flip":
        orig = so.conv3_backward
        monkeypatch.setattr(so, "conv3_backward", lambda x, w, dy: orig(x, w[:, :, ::-1], dy))
    else:
        monkeypatch.setattr(so, "upsample_backward", lambda dy, f: dy[..., ::f] if f > 1 else dy)
    net = tiny_net(so)
    x = inputs.uniform(11, (3, 9), -1, 1)
    target = inputs.uniform(12, (3, 3, 20), -1, 1)
    _, grads = net.backward(x, target)
    worst = 0.0
    for k in net.p:
        d = inputs.uniform(13, net.p[k].shape, -1, 1, stream=len(k))
        h = 1e-5
        base = net.p[k].copy()
        net.p[k] = base + h * d
        lp = net.loss(x, target)
        net.p[k] = base - h * d
        lm = net.loss(x, target)
        net.p[k] = base
        fd = (lp - lm) / (2 * h)
        worst = max(worst, abs(fd - float(np.sum(grads[k] * d))) / max(abs(fd), 1e-12))
    assert worst > 1e-4


def test_adam_first_step_and_bf16(so):
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 1e-3])
    m, v = np.zeros(3), np.zeros(3)
    so.adam_step(p, g, m, v, step=1, lr=0.1, eps=0.0)
    np.testing.assert_allclose(p, [0.9, -1.9, 2.9], rtol=0, atol=1e-15)  # first step = lr * sign(g)
    one = 1.0
    assert so.bf16_round(one) == 1.0
    assert so.bf16_round(1.0 + 2.0 ** -8) == 1.0            # tie, even mantissa kept
    assert so.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie, rounds up to even
    assert so.bf16_round(1.0 + 2.0 ** -8 + 2.0 ** -12) == 1.0 + 2.0 ** -7
    assert so.bf16_round(-3.0) == -3.0


def test_contracted_network_gradients_match_finite_differences(so):
    """With the moment contraction (output linear in the last six inputs)."""
    stages = [(4, 5, 2), (5, 12, 1)]
    sizes = {"W1": (6, 9), "b1": (6,), "W2": (6, 6), "b2": (6,), "W3": (4 * 5, 6), "b3": (20,)}
    for s, (ci, co, _) in enumerate(stages):
        sizes[f"C{s}"] = (co, ci, 3)
        sizes[f"c{s}"] = (co,)
    params = {k: inputs.uniform(4, v, -0.6, 0.6, stream=i) for i, (k, v) in enumerate(sizes.items())}
    net = so.Surrogate(params, 4, 5, stages, contract=6)
    x = inputs.uniform(11, (3, 9), -1, 1)
    target = inputs.uniform(12, (3, 2, 10), -1, 1)
    y, _ = net.forward(x)
    assert y.shape == (3, 2, 10)
    # exactly linear in the contracted inputs
    x2 = x.copy()
    x2[:, 3:] *= 2.0
    net_lin = so.Surrogate(params, 4, 5, stages, contract=6)
    y2 = np.einsum("nk,nkct->nct", x2[:, 3:], net_lin.forward(x)[1]["pre1"].reshape(3, 6, 2, 10))
    np.testing.assert_allclose(y2, 2 * y, rtol=1e-12, atol=1e-14)
    _, grads = net.backward(x, target)
    for k in net.p:
        d = inputs.uniform(13, net.p[k].shape, -1, 1, stream=len(k))
        h = 1e-5
        base = net.p[k].copy()
        net.p[k] = base + h * d
        lp = net.loss(x, target)
        net.p[k] = base - h * d
        lm = net.loss(x, target)
        net.p[k] = base
        fd = (lp - lm) / (2 * h)
        assert abs(fd - float(np.sum(grads[k] * d))) <= 1e-6 * max(abs(fd), 1e-12), k


def test_bf16_operand_mode_stays_close(so):
    """Rounding every product operand to bfloat16 (the tensor-core arithmetic) moves the output
    by no more than a few bfloat16 roundings (2^-9 relative each) along the layers, and the
    rounding itself is the identity on values already in bfloat16."""
    net = tiny_net(so)
    rounded = so.Surrogate(net.p, 4, 5, net.stages, bf16_operands=True)
    x = inputs.uniform(11, (3, 9), -1, 1)
    y, _ = net.forward(x)
    yr, _ = rounded.forward(x)
    rel = np.linalg.norm(yr - y) / np.linalg.norm(y)
    assert 0 < rel <= 3e-2
    xb = so.bf16_round(x)
    assert np.array_equal(so.bf16_round(xb), xb)
