"""A small residual CNN that corrects the fast reconstruction towards the direct one (the
learned extension beside the paper's method: the fast FBP's image plus a learned residual).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Network: six 3x3 convolutions (zero padding, stride 1) with channel counts 1 -> C -> ... ->
C -> 1, a ReLU after each but the last, and the input image added to the output:
    y = x + conv_6(relu(conv_5(... relu(conv_1(x)) ...))).
conv(x)[o][r][c] = b[o] + sum_{i, dy, dx} w[o][i][dy][dx] x[i][r + dy - 1][c + dx - 1]
(cross-correlation, as deep-learning convolutions are defined), x = 0 outside the image.
Loss: mean squared error against a target image.  Everything here is float64; gradients
are written out by hand (the chain rule through each step) and pinned by finite
differences in the tests.
"""
from __future__ import annotations

import numpy as np


def conv3x3(x, w, b) -> np.ndarray:
    """x [Ci][H][W], w [Co][Ci][3][3], b [Co] -> [Co][H][W]."""
    x = np.asarray(x, np.float64)
    Ci, H, W = x.shape
    xp = np.zeros((Ci, H + 2, W + 2))
    xp[:, 1:-1, 1:-1] = x
    out = np.zeros((w.shape[0], H, W)) + np.asarray(b, np.float64)[:, None, None]
    for dy in range(3):
        for dx in range(3):
            out += np.einsum("oi,ihw->ohw", w[:, :, dy, dx], xp[:, dy:dy + H, dx:dx + W])
    return out


def conv3x3_backward(x, w, gout):
    """Gradients of conv3x3 given dL/d(out) = gout: returns (dL/dx, dL/dw, dL/db)."""
    x = np.asarray(x, np.float64)
    Ci, H, W = x.shape
    xp = np.zeros((Ci, H + 2, W + 2))
    xp[:, 1:-1, 1:-1] = x
    gw = np.zeros_like(w, dtype=np.float64)
    gxp = np.zeros_like(xp)
    for dy in range(3):
        for dx in range(3):
            gw[:, :, dy, dx] = np.einsum("ohw,ihw->oi", gout, xp[:, dy:dy + H, dx:dx + W])
            gxp[:, dy:dy + H, dx:dx + W] += np.einsum("oi,ohw->ihw", w[:, :, dy, dx], gout)
    return gxp[:, 1:-1, 1:-1], gw, gout.sum(axis=(1, 2))


def init_params(channels: int = 32, layers: int = 6, seed: int = 0, scale: float = 1.0):
    """He-style normal weights (the last layer scaled down so the net starts near the
    identity), zero biases."""
    rng = np.random.default_rng(seed)
    dims = [1] + [channels] * (layers - 1) + [1]
    params = []
    for k in range(layers):
        ci, co = dims[k], dims[k + 1]
        std = np.sqrt(2.0 / (9 * ci)) * (0.1 if k == layers - 1 else 1.0) * scale
        params.append((rng.normal(0.0, std, (co, ci, 3, 3)), np.zeros(co)))
    return params


def forward(params, x):
    """y = x + net(x) for one image x [H][W]; returns (y, cache of layer inputs)."""
    h = np.asarray(x, np.float64)[None]
    cache = []
    for k, (w, b) in enumerate(params):
        cache.append(h)
        z = conv3x3(h, w, b)
        h = np.maximum(z, 0.0) if k < len(params) - 1 else z
    return x + h[0], cache


def loss_and_grads(params, x, target):
    """Mean squared error of forward(x) against target, and its gradients
    [(dw, db) per layer] and dL/dx."""
    y, cache = forward(params, x)
    r = y - target
    loss = float(np.mean(r * r))
    g = (2.0 / r.size) * r                       # dL/dy
    gx_skip = g
    gh = g[None]
    grads = [None] * len(params)
    for k in range(len(params) - 1, -1, -1):
        w, b = params[k]
        hin = cache[k]
        gin, gw, gb = conv3x3_backward(hin, w, gh)
        grads[k] = (gw, gb)
        if k > 0:
            gh = gin * (hin > 0.0)               # ReLU of the previous layer (hin = relu(z))
        else:
            gh = gin
    return loss, grads, gx_skip + gh[0]
