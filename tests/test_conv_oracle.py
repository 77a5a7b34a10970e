"""Pins of the FP64 layer reference used to check the warm-start kernels:
an independent scipy correlation for the forward pass, exact adjoint
identities for the gradients, and central finite differences."""
import numpy as np
import pytest
import scipy.signal as ss

from oracle import conv_oracle as C


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_conv_forward_matches_scipy_correlation():
    x = _rand((2, 9, 11, 3), 0)
    w = _rand((4, 3, 3, 3), 1)
    b = _rand(4, 2)
    out = C.conv3x3(x, w, b)
    for n in range(2):
        for co in range(4):
            ref = sum(ss.correlate2d(x[n, :, :, ci], w[co, :, :, ci], mode="same") for ci in range(3)) + b[co]
            assert np.abs(out[n, :, :, co] - ref).max() < 1e-12


def test_gradients_are_adjoints():
    x = _rand((2, 8, 6, 5), 3)
    w = _rand((7, 3, 3, 5), 4)
    dy = _rand((2, 8, 6, 7), 5)
    y = C.conv3x3(x, w)
    # <conv(x, w), dy> = <x, dgrad(dy, w)> = <w, wgrad(x, dy)>
    lhs = np.sum(y * dy)
    assert abs(lhs - np.sum(x * C.conv3x3_dgrad(dy, w))) < 1e-10 * abs(lhs)
    assert abs(lhs - np.sum(w * C.conv3x3_wgrad(x, dy))) < 1e-10 * abs(lhs)
    # pooling / upsampling adjoints
    a = _rand((1, 8, 6, 3), 6)
    c = _rand((1, 4, 3, 3), 7)
    assert abs(np.sum(C.avgpool2(a) * c) - np.sum(a * C.avgpool2_grad(c))) < 1e-12
    assert abs(np.sum(C.upsample2(c) * a) - np.sum(c * C.upsample2_grad(a))) < 1e-12


def test_two_layer_gradient_by_finite_differences():
    """loss = 1/2 ||conv(lrelu(conv(x, w1) + b1), w2)||^2: the chained
    reference gradients agree with central differences."""
    x = _rand((1, 6, 5, 2), 8)
    w1, b1 = 0.5 * _rand((3, 3, 3, 2), 9), 0.1 * _rand(3, 10)
    w2 = 0.5 * _rand((2, 3, 3, 3), 11)

    def loss(w1_, b1_, w2_):
        h = C.conv3x3(x, w1_, b1_)
        return 0.5 * np.sum(C.conv3x3(C.leaky_relu(h), w2_) ** 2)

    h = C.conv3x3(x, w1, b1)
    a = C.leaky_relu(h)
    y = C.conv3x3(a, w2)
    gw2 = C.conv3x3_wgrad(a, y)
    gh = C.leaky_relu_grad(h, C.conv3x3_dgrad(y, w2))
    gw1 = C.conv3x3_wgrad(x, gh)
    gb1 = C.bias_grad(gh)
    eps = 1e-6
    for arr, g, name in ((w1, gw1, "w1"), (b1, gb1, "b1"), (w2, gw2, "w2")):
        flat = arr.reshape(-1)
        for idx in np.random.default_rng(12).choice(flat.size, size=min(8, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp = loss(w1, b1, w2)
            flat[idx] = old - eps
            lm = loss(w1, b1, w2)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g.reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, g.reshape(-1)[idx])
