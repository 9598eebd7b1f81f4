"""Refining the recursive-filter coefficients against the direct FBP by gradient descent
through the adjoint kernels: the adjoint gradient with respect to the numerator against
central finite differences of the image-space loss, and a short fit that lowers the loss."""
import numpy as np
import pytest

import phantoms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    return t


def problem(fbp, torch, N, S, seed):
    K, M = phantoms.geometry_for(N)
    sino = phantoms.phantom_stack_torch(N, S, seed, "cuda", noise_i0=1e5)
    direct = torch.empty(S, N, N, device="cuda")
    fbp.fbp_direct_reconstruct(fbp.fbp_plan(N, K, M, S), sino, direct)
    torch.cuda.synchronize()
    return sino, direct


def test_numerator_gradient_matches_finite_differences(fbp, torch, coeff_table):
    from paper_2007_06289_gb300 import iir_fit, iir_fit_direct
    N = 64
    sino, direct = problem(fbp, torch, N, 4, 300)
    b, a = iir_fit.coefficients(N, 3, coeff_table)
    loss, g = iir_fit_direct.loss_and_grad_b(N, sino, direct, b, a)
    h = 1e-3
    for k in range(len(b)):
        d = np.zeros(len(b))
        d[k] = h
        lp, _ = iir_fit_direct.loss_and_grad_b(N, sino, direct, b + d, a)
        lm, _ = iir_fit_direct.loss_and_grad_b(N, sino, direct, b - d, a)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 2e-2 * np.abs(g).max() + 1e-9, (k, fd, g[k])


def test_fit_lowers_the_loss_against_direct_fbp(fbp, torch, coeff_table):
    from paper_2007_06289_gb300 import iir_fit, iir_fit_direct
    N = 64
    sino, direct = problem(fbp, torch, N, 8, 400)
    b0, a0 = iir_fit.coefficients(N, 3, coeff_table)
    b, a, losses = iir_fit_direct.fit_against_direct(N, sino, direct, b0, a0, steps=20)
    assert min(losses) < 0.95 * losses[0], losses
    assert np.abs(np.roots(np.concatenate([[1.0], a]))).max() < 1.0
    assert abs(b.sum()) <= 1e-9 * np.abs(b).sum()
