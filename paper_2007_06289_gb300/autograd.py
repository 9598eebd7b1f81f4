"""The fast reconstruction as a differentiable torch operation.

The reconstruction is linear in the sinogram (filter, resampling and back projection are
all linear), so its derivative is the operator itself and the backward pass is its adjoint:
``fbp_reconstruct_adjoint`` (the transposed back projection, the transposed resampling and
the symmetric filter, all in the library's kernels).  Both directions run through the C ABI;
nothing here computes.
"""
from __future__ import annotations

import torch

from . import binding as fbp


class _FastFBP(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sino, plan):
        img = torch.empty(plan.img_shape, device=sino.device, dtype=torch.float32)
        fbp.fbp_reconstruct(plan, sino.detach().contiguous(), img)
        ctx.plan = plan
        return img

    @staticmethod
    def backward(ctx, grad_img):
        plan = ctx.plan
        grad = torch.empty(plan.sino_shape, device=grad_img.device, dtype=torch.float32)
        fbp.fbp_reconstruct_adjoint(plan, grad_img.contiguous(), grad)
        return grad, None


def fast_fbp(sino: torch.Tensor, plan) -> torch.Tensor:
    """Images [batch][N][N] of sinograms [batch][K][M] (float32 CUDA), differentiable in
    the sinograms."""
    return _FastFBP.apply(sino, plan)


class FastFBP(torch.nn.Module):
    """Module form: owns a plan for `batch` slices of N x N from K angles x M bins."""

    def __init__(self, N: int, K: int, M: int, batch: int = 1, coeffs=None, fuse_k: int = 0):
        super().__init__()
        self.plan = fbp.fbp_plan(N, K, M, batch, coeffs, fuse_k)

    def forward(self, sino: torch.Tensor) -> torch.Tensor:
        return fast_fbp(sino, self.plan)
