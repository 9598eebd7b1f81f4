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

Storage precision.  The corrector is specified with bfloat16 weights and activations and
float32 accumulation.  With ``storage="bf16"`` the network keeps exactly those stored
values: the weights of the hidden 32 -> 32 layers and every hidden activation (after its
ReLU), and on the way back every hidden pre-activation gradient (after its ReLU mask), are
rounded to the nearest bfloat16; the first and last layers' weights, the input image and
the output stay as given.  All sums stay float64, so the only difference to a float32
accumulation is the accumulation's own rounding (and, rarely, a bfloat16 rounding decision
that this moves across a tie point).  With integer-valued parameters and images whose every
stored value is an integer of magnitude <= 256 and whose every sum stays below 2^24, both
storage modes and any float32 accumulation order give identical results.
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
            out += np.einsum("oi,ihw->ohw", w[:, :, dy, dx], xp[:, dy:dy + H, dx:dx + W],
                             optimize=True)
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
            gw[:, :, dy, dx] = np.einsum("ohw,ihw->oi", gout, xp[:, dy:dy + H, dx:dx + W],
                                         optimize=True)
            gxp[:, dy:dy + H, dx:dx + W] += np.einsum("oi,ohw->ihw", w[:, :, dy, dx], gout,
                                                      optimize=True)
    return gxp[:, 1:-1, 1:-1], gw, gout.sum(axis=(1, 2))


def bf16(x) -> np.ndarray:
    """Nearest bfloat16 of each value (the upper 16 bits of its IEEE float32, ties to even),
    returned as float64.  The value is rounded to float32 first."""
    v = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    u = v.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _stored(params, storage):
    """The weights as the network uses them: hidden 32 -> 32 layers rounded to bfloat16
    under storage="bf16"."""
    if storage == "f64":
        return params
    if storage != "bf16":
        raise ValueError(storage)
    L = len(params)
    return [(bf16(w) if 0 < k < L - 1 else w, b) for k, (w, b) in enumerate(params)]


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


def forward(params, x, storage: str = "f64"):
    """y = x + net(x) for one image x [H][W]; returns (y, cache of layer inputs).
    storage: "f64" (every value float64) or "bf16" (the stored precision, module docstring)."""
    ps = _stored(params, storage)
    h = np.asarray(x, np.float64)[None]
    cache = []
    for k, (w, b) in enumerate(ps):
        cache.append(h)
        z = conv3x3(h, w, b)
        if k < len(ps) - 1:
            h = np.maximum(z, 0.0)
            if storage == "bf16":
                h = bf16(h)
        else:
            h = z
    return x + h[0], cache


def backward(params, cache, gy, storage: str = "f64"):
    """Gradients [(dw, db) per layer] and dL/dx of a loss L given dL/dy = gy [H][W] and the
    cache of forward(params, x, storage).  Under storage="bf16" each hidden pre-activation
    gradient is rounded to bfloat16 after its ReLU mask, as it is stored."""
    ps = _stored(params, storage)
    gy = np.asarray(gy, np.float64)
    gh = gy[None]
    grads = [None] * len(ps)
    for k in range(len(ps) - 1, -1, -1):
        w, b = ps[k]
        hin = cache[k]
        gin, gw, gb = conv3x3_backward(hin, w, gh)
        grads[k] = (gw, gb)
        if k > 0:
            gh = gin * (hin > 0.0)               # ReLU of the previous layer (hin = relu(z))
            if storage == "bf16":
                gh = bf16(gh)
        else:
            gh = gin
    return grads, gy + gh[0]


def loss_and_grads(params, x, target, storage: str = "f64"):
    """Mean squared error of forward(x) against target, and its gradients
    [(dw, db) per layer] and dL/dx."""
    y, cache = forward(params, x, storage)
    r = y - target
    loss = float(np.mean(r * r))
    g = (2.0 / r.size) * r                       # dL/dy
    grads, gx = backward(params, cache, g, storage)
    return loss, grads, gx
