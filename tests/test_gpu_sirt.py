"""Algebraic reconstruction (SIRT on the fast Hough operators) and the fast Radon transform on
the GPU against the oracle.

Tolerances: the Hough-space data use the resampling's float32 positions and weights
(compared at 1e-6 of the largest value); SIRT iterates float32 sums of the exact operators,
compared with the float64 oracle after a few steps at 1e-5 of the largest pixel.
"""
import numpy as np
import pytest

import oracle.sirt as so
import phantoms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    return t


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("N", [2, 16, 64])
def test_hough_data_matches_oracle(fbp, torch, N):
    K, M = phantoms.geometry_for(N)
    rng = np.random.default_rng(N)
    sino = rng.normal(size=(2, K, M)).astype(np.float32)
    plan = fbp.fbp_plan(N, K, M, 2)
    lin = torch.full(plan.lin_shape, float("nan"), device="cuda")
    fbp.fbp_hough_data(plan, dev(torch, sino), lin)
    torch.cuda.synchronize()
    got = lin.cpu().numpy()
    for s in range(2):
        want = so.hough_data(sino[s].astype(np.float64), N)
        assert np.abs(got[s] - want).max() <= 1e-6 * np.abs(want).max()


def test_sirt_matches_oracle(fbp, torch):
    N, B, iters = 32, 2, 5
    K, M = phantoms.geometry_for(N)
    rng = np.random.default_rng(3)
    f_true = rng.normal(size=(B, N, N))
    b = np.stack([so.hough_project(f_true[s]) for s in range(B)]).astype(np.float32)
    b = b + (0.05 * rng.normal(size=b.shape) * (b != 0)).astype(np.float32)
    plan = fbp.fbp_plan(N, K, M, B)
    img = torch.zeros(plan.img_shape, device="cuda")
    fbp.fbp_sirt(plan, dev(torch, b), img, iters, 1.2)
    torch.cuda.synchronize()
    got = img.cpu().numpy()
    for s in range(B):
        want = so.sirt(b[s].astype(np.float64), N, iters, 1.2)
        assert np.abs(got[s] - want).max() <= 1e-5 * np.abs(want).max()


def test_sirt_recovers_the_image_from_consistent_data(fbp, torch):
    # data from the GPU projector of a phantom image; the error falls with the iterations
    N = 64
    K, M = phantoms.geometry_for(N)
    plan = fbp.fbp_plan(N, K, M, 1)
    gen = torch.Generator(device="cuda").manual_seed(4)
    f_true = torch.rand(plan.img_shape, device="cuda", generator=gen)
    b = torch.empty(plan.lin_shape, device="cuda")
    fbp.fbp_hough_project(plan, f_true, b)
    img = torch.zeros(plan.img_shape, device="cuda")
    errs = []
    for _ in range(4):
        fbp.fbp_sirt(plan, b, img, 50, 1.5)
        errs.append(float(torch.linalg.norm(img - f_true) / torch.linalg.norm(f_true)))
    assert all(e1 < e0 for e0, e1 in zip(errs, errs[1:])), errs
    assert errs[-1] < 0.5 * errs[0], errs


def test_sirt_chunks_equal_single_slices(fbp, torch):
    N, B = 32, 3
    K, M = phantoms.geometry_for(N)
    rng = np.random.default_rng(5)
    b = dev(torch, np.stack([so.hough_project(rng.normal(size=(N, N))) for _ in range(B)]))
    plan = fbp.fbp_plan(N, K, M, B)
    fbp.fbp_set_chunk(plan, 2)
    img = torch.zeros(plan.img_shape, device="cuda")
    fbp.fbp_sirt(plan, b, img, 3, 1.0)
    one = fbp.fbp_plan(N, K, M, 1)
    for s in range(B):
        ref = torch.zeros(one.img_shape, device="cuda")
        fbp.fbp_sirt(one, b[s:s + 1].contiguous(), ref, 3, 1.0)
        torch.cuda.synchronize()
        assert torch.equal(img[s:s + 1], ref)


def test_sirt_rejects_bad_relaxation(fbp, torch):
    N = 8
    K, M = phantoms.geometry_for(N)
    plan = fbp.fbp_plan(N, K, M, 1)
    b = torch.zeros(plan.lin_shape, device="cuda")
    img = torch.zeros(plan.img_shape, device="cuda")
    for lam in (0.0, 2.0, -1.0, float("nan")):
        with pytest.raises(RuntimeError):
            fbp.fbp_sirt(plan, b, img, 1, lam)


@pytest.mark.parametrize("N", [2, 16, 64])
def test_fast_radon_matches_oracle(fbp, torch, N):
    import oracle.radon as orad
    K, M = phantoms.geometry_for(N)
    rng = np.random.default_rng(N + 9)
    img = rng.random(size=(2, N, N)).astype(np.float32)
    plan = fbp.fbp_plan(N, K, M, 2)
    sino = torch.full(plan.sino_shape, float("nan"), device="cuda")
    fbp.fbp_radon(plan, dev(torch, img), sino)
    torch.cuda.synchronize()
    got = sino.cpu().numpy()
    for s in range(2):
        want = orad.fast_radon(img[s].astype(np.float64), K, M)
        assert np.abs(got[s] - want).max() <= 1e-5 * np.abs(want).max()


def test_fast_radon_keeps_the_mass_at_512(fbp, torch):
    N = 512
    K, M = phantoms.geometry_for(N)
    plan = fbp.fbp_plan(N, K, M, 2)
    gen = torch.Generator(device="cuda").manual_seed(6)
    img = torch.rand(plan.img_shape, device="cuda", generator=gen)
    sino = torch.empty(plan.sino_shape, device="cuda")
    fbp.fbp_radon(plan, img, sino)
    torch.cuda.synchronize()
    mass = sino.double().sum(dim=2)
    total = img.double().sum(dim=(1, 2))
    assert float((mass / total[:, None] - 1).abs().max()) < 1e-2


def test_radon_and_hough_data_chunks_equal_single_slices(fbp, torch):
    N, B = 32, 3
    K, M = phantoms.geometry_for(N)
    rng = np.random.default_rng(8)
    img = dev(torch, rng.random(size=(B, N, N)))
    sino = dev(torch, rng.normal(size=(B, K, M)))
    plan = fbp.fbp_plan(N, K, M, B)
    fbp.fbp_set_chunk(plan, 2)
    rad = torch.empty(plan.sino_shape, device="cuda")
    hd = torch.empty(plan.lin_shape, device="cuda")
    fbp.fbp_radon(plan, img, rad)
    fbp.fbp_hough_data(plan, sino, hd)
    one = fbp.fbp_plan(N, K, M, 1)
    for s in range(B):
        r1 = torch.empty(one.sino_shape, device="cuda")
        h1 = torch.empty(one.lin_shape, device="cuda")
        fbp.fbp_radon(one, img[s:s + 1].contiguous(), r1)
        fbp.fbp_hough_data(one, sino[s:s + 1].contiguous(), h1)
        torch.cuda.synchronize()
        assert torch.equal(rad[s:s + 1], r1)
        assert torch.equal(hd[s:s + 1], h1)


def test_sirt_with_no_iterations_leaves_the_image(fbp, torch):
    N = 16
    K, M = phantoms.geometry_for(N)
    plan = fbp.fbp_plan(N, K, M, 1)
    b = torch.ones(plan.lin_shape, device="cuda")
    img = torch.randn(plan.img_shape, device="cuda")
    before = img.clone()
    fbp.fbp_sirt(plan, b, img, 0, 1.0)
    torch.cuda.synchronize()
    assert torch.equal(img, before)
