"""FP64 CPU reference of the warm-start network's layers (TEST INFRASTRUCTURE
ONLY: imported by the tests, never by the product path).

The learned warm start maps the medium and forcing to an initial guess for
the CG solve of eq. (amat_sym).  Its layers are 3x3 convolutions with zero
padding (stride 1), per-channel bias, leaky ReLU, 2x2 average pooling,
nearest-neighbour 2x upsampling and channel concatenation, on NHWC tensors.
Each function below is the plain definition written out with numpy; the
gradients are the exact adjoints (pinned in tests/test_conv_oracle.py by
inner-product identities, an independent scipy correlation and finite
differences).
"""
from __future__ import annotations

import numpy as np

LEAK = 0.1


def conv3x3(x, w, b=None):
    """out[n, y, x, co] = sum_{ky, kx, ci} w[co, ky, kx, ci] * x[n, y+ky-1, x+kx-1, ci] (+ b[co]),
    x zero outside the image.  x: [N, H, W, Ci], w: [Co, 3, 3, Ci]."""
    N, H, W, Ci = x.shape
    Co = w.shape[0]
    xp = np.zeros((N, H + 2, W + 2, Ci))
    xp[:, 1:-1, 1:-1, :] = x
    out = np.zeros((N, H, W, Co))
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, ky:ky + H, kx:kx + W, :]                  # [N, H, W, Ci]
            out += patch @ w[:, ky, kx, :].T                        # [Ci] x [Ci, Co]
    if b is not None:
        out += b
    return out


def conv3x3_dgrad(dy, w):
    """d(loss)/dx of conv3x3 for d(loss)/d(out) = dy: sum over the output pixels
    that read x[n, y, x, ci]."""
    N, H, W, Co = dy.shape
    Ci = w.shape[3]
    dxp = np.zeros((N, H + 2, W + 2, Ci))
    for ky in range(3):
        for kx in range(3):
            dxp[:, ky:ky + H, kx:kx + W, :] += dy @ w[:, ky, kx, :]
    return dxp[:, 1:-1, 1:-1, :]


def conv3x3_wgrad(x, dy):
    """d(loss)/dw[co, ky, kx, ci] = sum_{n, y, x} dy[n, y, x, co] * x[n, y+ky-1, x+kx-1, ci]."""
    N, H, W, Ci = x.shape
    Co = dy.shape[3]
    xp = np.zeros((N, H + 2, W + 2, Ci))
    xp[:, 1:-1, 1:-1, :] = x
    dw = np.zeros((Co, 3, 3, Ci))
    dyf = dy.reshape(-1, Co)
    for ky in range(3):
        for kx in range(3):
            dw[:, ky, kx, :] = dyf.T @ xp[:, ky:ky + H, kx:kx + W, :].reshape(-1, Ci)
    return dw


def bias_grad(dy):
    return dy.reshape(-1, dy.shape[-1]).sum(axis=0)


def leaky_relu(x):
    return np.where(x > 0, x, LEAK * x)


def leaky_relu_grad(x, dy):
    return np.where(x > 0, dy, LEAK * dy)


def avgpool2(x):
    N, H, W, C = x.shape
    return x.reshape(N, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def avgpool2_grad(dy):
    return 0.25 * np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2)


def upsample2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample2_grad(dy):
    N, H, W, C = dy.shape
    return dy.reshape(N, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))
