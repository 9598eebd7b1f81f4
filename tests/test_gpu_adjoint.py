"""Adjoints on the GPU against the oracle's adjoints, the adjoint identity, and the torch
autograd wrapper.

Tolerances: the transposed back projection is bit for bit the oracle's float32 transposed
stage recursion (fixed float32 sums); the transposed resampling gathers in its own fixed
order with float32 weights and positions (like the forward resampling), so it and the whole
adjoint are compared with the float64 oracle at 2e-5 of the largest value, and with
themselves bit for bit from run to run.
"""
import numpy as np
import pytest

import oracle
import phantoms

pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    return t


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("N", [2, 4, 8, 16, 64, 128, 256])
def test_backprojection_adjoint_bit_exact(fbp, torch, N):
    rng = np.random.default_rng(N)
    g = rng.normal(size=(2, N, N)).astype(np.float32)
    K, M = phantoms.geometry_for(N)
    plan = fbp.fbp_plan(N, K, M, 2)
    lin = torch.full(plan.lin_shape, float("nan"), device="cuda")
    fbp.fbp_fht_backproject_adjoint(plan, dev(torch, g), lin)
    torch.cuda.synchronize()
    got = lin.cpu().numpy()
    for b in range(2):
        want = oracle.fht_backproject_adjoint(g[b])
        np.testing.assert_array_equal(got[b], want)


@pytest.mark.parametrize("N", [1024, 2048])
def test_backprojection_adjoint_bit_exact_large(fbp, torch, N):
    # N = 1024: two launches of five stages; N = 2048: three launches (4 + 4 + 3), the
    # middle one reading and writing partially written level arrays
    rng = np.random.default_rng(N + 7)
    g = rng.normal(size=(1, N, N)).astype(np.float32)
    K, M = phantoms.geometry_for(N)
    plan = fbp.fbp_plan(N, K, M, 1)
    lin = torch.full(plan.lin_shape, float("nan"), device="cuda")
    fbp.fbp_fht_backproject_adjoint(plan, dev(torch, g), lin)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(lin.cpu().numpy()[0], oracle.fht_backproject_adjoint(g[0]))


def test_backprojection_adjoint_integer_inputs_exact(fbp, torch):
    N = 256
    rng = np.random.default_rng(9)
    g = rng.integers(-1024, 1024, size=(1, N, N)).astype(np.float32)
    K, M = phantoms.geometry_for(N)
    plan = fbp.fbp_plan(N, K, M, 1)
    lin = torch.empty(plan.lin_shape, device="cuda")
    fbp.fbp_fht_backproject_adjoint(plan, dev(torch, g), lin)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(lin.cpu().numpy()[0],
                                  oracle.fht_backproject_adjoint(g[0].astype(np.float64),
                                                                 brute=True))


@pytest.mark.parametrize("N", [2, 8, 16, 64])
def test_resampling_adjoint_matches_oracle(fbp, torch, N):
    # N = 2: K = 3, a partial last group of sinogram rows and the mirrored row-0 reads
    rng = np.random.default_rng(N + 1)
    K, M = phantoms.geometry_for(N)
    lb = rng.normal(size=(1, 4, N, 2 * N)).astype(np.float32)
    plan = fbp.fbp_plan(N, K, M, 1)
    out = torch.full(plan.sino_shape, float("nan"), device="cuda")
    fbp.fbp_resample_st_adjoint(plan, dev(torch, lb), out)
    torch.cuda.synchronize()
    want = oracle.linogram_adjoint(lb[0].astype(np.float64), N, K, M)
    assert np.abs(out.cpu().numpy()[0] - want).max() <= TOL * np.abs(want).max()


def test_reconstruct_adjoint_matches_oracle(fbp, torch, coeff_table):
    N = 64
    K, M = phantoms.geometry_for(N)
    e = next(e for e in coeff_table["entries"] if e["N"] == N and e["order"] == 3)
    b, a = list(e["b"]), list(e["a"])
    rng = np.random.default_rng(2)
    g = rng.normal(size=(2, N, N)).astype(np.float32)
    plan = fbp.fbp_plan(N, K, M, 2, (b, a))
    out = torch.empty(plan.sino_shape, device="cuda")
    fbp.fbp_reconstruct_adjoint(plan, dev(torch, g), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for s in range(2):
        want = oracle.fast_fbp_adjoint(g[s].astype(np.float64), N, K, M, b, a)
        assert np.abs(got[s] - want).max() <= TOL * np.abs(want).max()


def test_adjoint_is_reproducible_bit_for_bit(fbp, torch):
    # no atomics anywhere in the adjoint: two runs agree exactly (N = 512, 3 slices)
    N, B = 512, 3
    K, M = phantoms.geometry_for(N)
    plan = fbp.fbp_plan(N, K, M, B)
    gen = torch.Generator(device="cuda").manual_seed(11)
    y = torch.randn(plan.img_shape, device="cuda", generator=gen)
    r1 = torch.empty(plan.sino_shape, device="cuda")
    r2 = torch.full(plan.sino_shape, float("nan"), device="cuda")
    fbp.fbp_reconstruct_adjoint(plan, y, r1)
    fbp.fbp_reconstruct_adjoint(plan, y, r2)
    torch.cuda.synchronize()
    assert torch.equal(r1, r2)


def test_adjoint_identity_batch_of_512(fbp, torch):
    # <R x, y> = <x, R^T y> for the GPU operator pair, B = 4 slices of N = 512
    N, B = 512, 4
    K, M = phantoms.geometry_for(N)
    plan = fbp.fbp_plan(N, K, M, B)
    gen = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn(plan.sino_shape, device="cuda", generator=gen)
    y = torch.randn(plan.img_shape, device="cuda", generator=gen)
    rx = torch.empty(plan.img_shape, device="cuda")
    rty = torch.empty(plan.sino_shape, device="cuda")
    fbp.fbp_reconstruct(plan, x, rx)
    fbp.fbp_reconstruct_adjoint(plan, y, rty)
    torch.cuda.synchronize()
    lhs = float((rx.double() * y.double()).sum())
    rhs = float((x.double() * rty.double()).sum())
    scale = float((rx.double().abs() * y.double().abs()).sum())
    assert abs(lhs - rhs) <= 1e-5 * scale


def test_autograd_gradient_is_the_adjoint(fbp, torch):
    from paper_2007_06289_gb300 import autograd as fa
    N, B = 128, 2
    K, M = phantoms.geometry_for(N)
    layer = fa.FastFBP(N, K, M, B)
    sino = phantoms.phantom_stack_torch(N, B, 11, "cuda").requires_grad_(True)
    w = torch.randn(B, N, N, device="cuda", generator=torch.Generator(device="cuda").manual_seed(1))
    img = layer(sino)
    ref = torch.empty(layer.plan.img_shape, device="cuda")
    fbp.fbp_reconstruct(layer.plan, sino.detach(), ref)
    assert torch.equal(img.detach(), ref)
    (img * w).sum().backward()
    adj = torch.empty(layer.plan.sino_shape, device="cuda")
    fbp.fbp_reconstruct_adjoint(layer.plan, w, adj)
    torch.cuda.synchronize()
    assert torch.allclose(sino.grad, adj, rtol=0, atol=1e-6 * float(adj.abs().max()))
    # directional derivatives (the operator is linear, so a finite difference along v is
    # R v exactly up to rounding): <grad, v> = <w, R v> for 64 random directions
    gen = torch.Generator(device="cuda").manual_seed(2)
    for _ in range(64):
        v = torch.randn(layer.plan.sino_shape, device="cuda", generator=gen)
        with torch.no_grad():
            rv = layer(v)
        lhs = float((sino.grad.double() * v.double()).sum())
        rhs = float((w.double() * rv.double()).sum())
        assert abs(lhs - rhs) <= 1e-4 * float((w.double().abs() * rv.double().abs()).sum())


def test_hough_projector_is_the_transposed_back_projection(fbp, torch):
    N, B = 128, 2
    K, M = phantoms.geometry_for(N)
    plan = fbp.fbp_plan(N, K, M, B)
    gen = torch.Generator(device="cuda").manual_seed(8)
    f = torch.randn(plan.img_shape, device="cuda", generator=gen)
    lin = torch.randn(plan.lin_shape, device="cuda", generator=gen)
    p1 = torch.empty(plan.lin_shape, device="cuda")
    p2 = torch.empty(plan.lin_shape, device="cuda")
    hl = torch.empty(plan.img_shape, device="cuda")
    fbp.fbp_hough_project(plan, f, p1)
    fbp.fbp_fht_backproject_adjoint(plan, f, p2)
    fbp.fbp_fht_backproject(plan, lin.clone(), hl)
    torch.cuda.synchronize()
    assert torch.equal(p1, p2)
    lhs = float((p1.double() * lin.double()).sum())
    rhs = float((f.double() * hl.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * float((p1.double().abs() * lin.double().abs()).sum())
    # a single pixel projects to 1 along each of its dyadic lines: N entries per quarter
    one = torch.zeros(plan.img_shape, device="cuda")
    one[0, 37, 90] = 1.0
    fbp.fbp_hough_project(plan, one, p1)
    torch.cuda.synchronize()
    assert float(p1[0].sum()) == 4 * N and int((p1[0] != 0).sum()) == 4 * N
