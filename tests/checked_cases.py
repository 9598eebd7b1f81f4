"""Parity cases run against the bounds-checked library (libfbp_checked.so, FBP_BOUNDS_CHECK):
every pipeline kernel range-checks its accesses there, so these small cases also assert that
the status word stays clear -- no index left its buffer or Hough tile.  The last case
corrupts one geometry row through the checked build's test hook and expects the kernels to
reject it (status FBP_ERR_INTERNAL, cleared by the read).

Not collected on its own (the file name does not start with test_): tests/test_gpu_checked.py
runs it in a subprocess with FBP_LIBRARY pointing at the checked library.
"""
import os

import numpy as np
import pytest

import oracle
import phantoms
from paper_2007_06289_gb300 import binding as fbp
from paper_2007_06289_gb300 import iir_fit

pytestmark = pytest.mark.gpu
FBP_ERR_INTERNAL = 7


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    assert fbp.load_library()._name == os.environ["FBP_LIBRARY"]
    assert hasattr(fbp.load_library(), "fbp_check_set_row_angle")
    return t


@pytest.mark.parametrize("N,fuse_k", [(8, 0), (64, 0), (128, 0), (128, 3), (256, 0), (256, 2),
                                      (256, 6), (512, 0)])
def test_fht_bit_exact_and_in_bounds(torch, N, fuse_k):
    rng = np.random.default_rng(N + fuse_k)
    lin = rng.normal(size=(2, 4, N, 2 * N)).astype(np.float32)
    plan = fbp.fbp_plan(N, 8, 8, 2, None, fuse_k)
    img = torch.empty(plan.img_shape, device="cuda")
    fbp.fbp_fht_backproject(plan, torch.from_numpy(lin).cuda(), img)
    assert fbp.fbp_last_device_error(plan) == 0
    for s in range(2):
        assert np.array_equal(img[s].cpu().numpy(), oracle.fht_backproject(lin[s]))


@pytest.mark.parametrize("N", [64, 256])
def test_pipeline_matches_oracle_and_in_bounds(torch, N):
    K, M = phantoms.geometry_for(N)
    b, a = iir_fit.coefficients(N, 3)
    sino = phantoms.phantom_stack_torch(N, 2, 77, "cuda", noise_i0=1e5)
    plan = fbp.fbp_plan(N, K, M, 2, (list(b), list(a)))
    img = torch.empty(plan.img_shape, device="cuda")
    fbp.fbp_reconstruct(plan, sino, img)
    lin = torch.empty(plan.lin_shape, device="cuda")
    filt = torch.empty(plan.sino_shape, device="cuda")
    fbp.fbp_filter_iir(plan, sino, filt)
    fbp.fbp_resample_st(plan, filt, lin)
    assert fbp.fbp_last_device_error(plan) == 0
    want = oracle.fast_fbp(sino[1].cpu().numpy().astype(np.float64), N, b, a)
    got = img[1].cpu().numpy()
    assert np.abs(got - want).max() <= 1e-5 * (want.max() - want.min())


def test_ragged_volume_in_bounds(torch):
    items = []
    for i, N in enumerate([64, 128, 64, 256]):
        K, M = phantoms.geometry_for(N)
        sino = phantoms.phantom_stack_torch(N, 1, 300 + i, "cuda")[0].contiguous()
        items.append((N, sino, torch.zeros((N, N), device="cuda")))
    vol = fbp.fbp_volume_create(items)
    vol.run()
    torch.cuda.synchronize()
    for N, sino, img in items:
        K, M = sino.shape
        plan = fbp.fbp_plan(N, K, M, 1)
        one = torch.empty(plan.img_shape, device="cuda")
        fbp.fbp_reconstruct(plan, sino[None].contiguous(), one)
        assert fbp.fbp_last_device_error(plan) == 0
        assert torch.equal(img, one[0])


def test_rejected_geometry_row_sets_the_status_word(torch):
    N = 64
    K, M = phantoms.geometry_for(N)
    sino = phantoms.phantom_stack_torch(N, 1, 5, "cuda")
    plan = fbp.fbp_plan(N, K, M, 1)
    img = torch.empty(plan.img_shape, device="cuda")
    fbp.fbp_reconstruct(plan, sino, img)
    assert fbp.fbp_last_device_error(plan) == 0
    fbp.fbp_check_set_row_angle(plan, 1, 5, K + 3)        # angle row past the sinogram
    fbp.fbp_reconstruct(plan, sino, img)
    assert fbp.fbp_last_device_error(plan) == FBP_ERR_INTERNAL
    assert fbp.fbp_last_device_error(plan) == 0            # the read cleared it
    assert torch.isfinite(img).all()
    lin = torch.empty(plan.lin_shape, device="cuda")
    filt = torch.empty(plan.sino_shape, device="cuda")
    fbp.fbp_filter_iir(plan, sino, filt)
    fbp.fbp_resample_st(plan, filt, lin)
    assert fbp.fbp_last_device_error(plan) == FBP_ERR_INTERNAL
    assert float(lin[0, 1, 5].abs().max()) == 0.0          # the rejected row is zeros
