"""Learned residual corrector for the fast reconstruction: y = x + net(x), six 3x3
convolutions (1 -> 32 x 5 -> 1 channels), trained on pairs of fast and direct-FBP images.

All arithmetic runs in the library's kernels (fbp_cnn_forward / fbp_cnn_backward); this
module holds the parameters, the workspaces, a torch.autograd.Function so that torch
optimisers can train them, and a small training loop.
"""
from __future__ import annotations

import math
import warnings

import numpy as np
import torch

from . import binding as fbp

CHANNELS = 32
LAYERS = 6


def init_params(seed: int = 0, scale: float = 1.0) -> np.ndarray:
    """He-normal weights (the last layer scaled by 0.1, so the corrector starts close to the
    identity), zero biases; fp32, in the library's parameter layout."""
    rng = np.random.default_rng(seed)
    dims = [1] + [CHANNELS] * (LAYERS - 1) + [1]
    out = []
    for k in range(LAYERS):
        ci, co = dims[k], dims[k + 1]
        std = math.sqrt(2.0 / (9 * ci)) * (0.1 if k == LAYERS - 1 else 1.0) * scale
        out.append(rng.normal(0.0, std, co * ci * 9))
        out.append(np.zeros(co))
    flat = np.concatenate(out).astype(np.float32)
    assert flat.size == fbp.fbp_cnn_param_count()
    return flat


class _Workspaces:
    def __init__(self):
        self._ws = {}

    def get(self, N, B, train, device):
        key = (N, B, bool(train), str(device))
        if key not in self._ws:
            nbytes = fbp.fbp_cnn_workspace_bytes(N, B, train)
            self._ws[key] = torch.empty(nbytes, dtype=torch.uint8, device=device)
        return self._ws[key]


_WS = _Workspaces()


class _CorrectorFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, x):
        B, N = x.shape[0], x.shape[-1]
        ws = _WS.get(N, B, True, x.device)
        y = torch.empty_like(x)
        xc = x.detach().contiguous()
        fbp.fbp_cnn_forward(params.detach(), xc, y, ws, train=True)
        ctx.save_for_backward(params, xc)
        ctx.ws = ws
        return y

    @staticmethod
    def backward(ctx, gy):
        params, x = ctx.saved_tensors
        g = torch.empty_like(params)
        fbp.fbp_cnn_backward(params.detach(), x, gy.contiguous(), g, ctx.ws)
        return g, None


def correct(params: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    """Differentiable in `params` (the gradient with respect to x is not provided)."""
    return _CorrectorFn.apply(params, x)


def infer(params: torch.Tensor, x: torch.Tensor, fallback: bool = False) -> torch.Tensor:
    """Inference without keeping activations.

    fallback=True: read the corrector's status word after the call (this synchronises the
    device).  If it is not clear -- a bounded wait in the corrector's kernels expired, or in
    the bounds-checked library a range check failed -- the output cannot be trusted, and the
    plain fast reconstruction x itself is returned (a copy, with a warning): the method
    without its corrector.  The status word is the process's, shared by every corrector
    call, so concurrent calls on other streams can trip it too."""
    B, N = x.shape[0], x.shape[-1]
    y = torch.empty_like(x)
    xc = x.contiguous()
    fbp.fbp_cnn_forward(params, xc, y, _WS.get(N, B, False, x.device), train=False)
    if fallback:
        status = fbp.fbp_cnn_last_error()
        if status != 0:
            warnings.warn(f"corrector status {status} ({fbp.fbp_status_str(status)}): "
                          "returning the uncorrected fast reconstruction", RuntimeWarning)
            return xc.clone()
    return y


def train(fast: torch.Tensor, target: torch.Tensor, steps: int = 300, batch: int = 4,
          lr: float = 1e-3, seed: int = 0) -> tuple[torch.Tensor, list[float]]:
    """Fit the corrector so that correct(fast) approaches target (mean squared error, Adam).
    fast, target: [S][N][N] float32 CUDA.  Returns (params, losses)."""
    dev = fast.device
    params = torch.tensor(init_params(seed), device=dev, requires_grad=True)
    opt = torch.optim.Adam([params], lr=lr)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    S = fast.shape[0]
    for _ in range(steps):
        idx = torch.randperm(S, generator=gen)[:batch].to(dev)
        y = correct(params, fast[idx])
        loss = torch.mean((y - target[idx]) ** 2)
        opt.zero_grad()
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    return params.detach(), losses
