"""Refining the recursive-filter coefficients against the direct FBP, in image space, by
gradient descent through the library's adjoint kernels.

The host fit (``iir_fit``) matches the filter's frequency response to the ideal ramp.  What
matters in the end is the reconstruction, so this module minimises instead
    loss(b, a) = mean over pixels and slices of (R_{b,a}(p) - D(p))^2,
R_{b,a} the fast reconstruction with coefficients (b, a) and D the direct FBP, over a set of
sinograms p.

Gradients.  R is linear in the filtered sinogram: R_{b,a}(p) = H L F_{b,a} p.  With the
image residual r = R - D, u = L^T H^T (2 r / n) (``fbp_fht_backproject_adjoint`` then
``fbp_resample_st_adjoint``) is the gradient of the loss with respect to the filtered
sinogram, and since F_{b,a} = sum_k b_k F_{e_k,a} is linear in b,
    d loss / d b_k = <u, F_{e_k,a} p>,
one filtering of p per coefficient (``fbp_filter_iir`` with numerator e_k).  The feedback
coefficients enter non-linearly; they are parameterised by reflection coefficients
k_i = 0.99999 tanh(x_i) (every trial filter stable) and their gradient is taken by central
differences of the loss.  The numerator keeps sum(b) = 0 (the gradient is projected).
Steps are Adam's.  Everything runs in the library's kernels; this module only orchestrates.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as fbp
from .iir_fit import KMAX, poly_to_reflection, reflection_to_poly


class _Problem:
    def __init__(self, N, sinos, target):
        self.N = N
        self.sinos = sinos.contiguous()
        self.target = target.contiguous()
        self.S, self.K, self.M = sinos.shape
        self.img = torch.empty_like(target)

    def plan(self, b, a):
        return fbp.fbp_plan(self.N, self.K, self.M, self.S, (list(map(float, b)), list(map(float, a))))

    def loss(self, b, a, plan=None):
        plan = plan or self.plan(b, a)
        fbp.fbp_reconstruct(plan, self.sinos, self.img)
        r = self.img - self.target
        return float(torch.mean(r.double() ** 2)), r, plan

    def grad_b(self, b, a, r, plan):
        """Adjoint-based gradient of the loss with respect to b."""
        n = r.numel()
        lin = torch.empty(plan.lin_shape, device=r.device)
        u = torch.empty(plan.sino_shape, device=r.device)
        fbp.fbp_fht_backproject_adjoint(plan, (2.0 / n) * r, lin)
        fbp.fbp_resample_st_adjoint(plan, lin, u)
        g = np.zeros(len(b))
        fk = torch.empty_like(self.sinos)
        for k in range(len(b)):
            e = np.zeros(len(b))
            e[k] = 1.0
            fbp.fbp_filter_iir(self.plan(e, a), self.sinos, fk)
            g[k] = float(torch.sum(u.double() * fk.double()))
        return g


def loss_and_grad_b(N, sinos, target, b, a):
    """(loss, d loss / d b) at (b, a): the adjoint path, exposed for checking."""
    pr = _Problem(N, sinos, target)
    loss, r, plan = pr.loss(b, a)
    return loss, pr.grad_b(b, a, r, plan)


def fit_against_direct(N, sinos, target, b0, a0, steps: int = 40, lr_b: float = 2e-3,
                       lr_x: float = 2e-2, fd: float = 1e-3):
    """Adam on (b, x) from (b0, a0).  sinos [S][K][M], target [S][N][N]: float32 CUDA.
    Returns (b, a, losses); losses[0] is the starting loss."""
    pr = _Problem(N, sinos, target)
    b = np.array(b0, dtype=np.float64)
    x = np.arctanh(np.clip(poly_to_reflection(np.asarray(a0, np.float64)) / KMAX, -0.999999, 0.999999))
    params = np.concatenate([b, x])
    m1 = np.zeros_like(params)
    m2 = np.zeros_like(params)
    lr = np.concatenate([np.full(b.size, lr_b), np.full(x.size, lr_x)])
    losses = []
    best = None
    for it in range(steps + 1):
        b, x = params[:b.size], params[b.size:]
        a = reflection_to_poly(KMAX * np.tanh(x))
        loss, r, plan = pr.loss(b, a)
        losses.append(loss)
        if best is None or loss < best[0]:
            best = (loss, b.copy(), a.copy())
        if it == steps:
            break
        gb = pr.grad_b(b, a, r, plan)
        gb -= gb.mean()                             # stay on sum(b) = 0
        gx = np.zeros(x.size)
        for i in range(x.size):
            d = np.zeros(x.size)
            d[i] = fd
            lp = pr.loss(b, reflection_to_poly(KMAX * np.tanh(x + d)))[0]
            lm = pr.loss(b, reflection_to_poly(KMAX * np.tanh(x - d)))[0]
            gx[i] = (lp - lm) / (2 * fd)
        g = np.concatenate([gb, gx])
        m1 = 0.9 * m1 + 0.1 * g
        m2 = 0.999 * m2 + 0.001 * g * g
        step = lr * (m1 / (1 - 0.9 ** (it + 1))) / (np.sqrt(m2 / (1 - 0.999 ** (it + 1))) + 1e-12)
        params = params - step
        params[:b.size] -= params[:b.size].mean()
    return best[1], best[2], losses
