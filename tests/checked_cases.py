"""Parity cases run against the bounds-checked library (libfbp_checked.so, FBP_BOUNDS_CHECK):
every kernel of the reconstruction, its adjoints, SIRT and the corrector range-checks its
accesses there, so these small cases also assert that the status words stay clear -- no
index left its buffer or Hough tile.  Two cases use the checked build's test hooks: one
makes the corrector's last layer see fewer images than the call has (its status word then
reads FBP_ERR_INTERNAL and the later images are left unwritten), the last corrupts one
geometry row and expects the kernels to reject it (status FBP_ERR_INTERNAL, cleared by the
read).

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


@pytest.mark.parametrize("N", [8, 64, 256])
def test_adjoints_match_oracle_and_in_bounds(torch, N):
    # N = 256: two launches of the fused transposed stages (5 + 3), the second reading the
    # first's partially written level arrays
    rng = np.random.default_rng(N + 40)
    K, M = phantoms.geometry_for(N)
    plan = fbp.fbp_plan(N, K, M, 2)
    g = rng.normal(size=(2, N, N)).astype(np.float32)
    lin = torch.full(plan.lin_shape, float("nan"), device="cuda")
    fbp.fbp_fht_backproject_adjoint(plan, torch.from_numpy(g).cuda(), lin)
    lb = rng.normal(size=plan.lin_shape).astype(np.float32)
    pb = torch.full(plan.sino_shape, float("nan"), device="cuda")
    fbp.fbp_resample_st_adjoint(plan, torch.from_numpy(lb).cuda(), pb)
    assert fbp.fbp_last_device_error(plan) == 0
    got_lin, got_pb = lin.cpu().numpy(), pb.cpu().numpy()
    for s in range(2):
        assert np.array_equal(got_lin[s], oracle.fht_backproject_adjoint(g[s]))
    want = oracle.linogram_adjoint(lb[1].astype(np.float64), N, K, M)
    assert np.abs(got_pb[1] - want).max() <= 2e-5 * np.abs(want).max()


def test_sirt_matches_oracle_and_in_bounds(torch):
    # the residual form of the last transposed launch (data and weights read on the way out)
    import oracle.sirt as so
    N, B, iters = 32, 2, 3
    K, M = phantoms.geometry_for(N)
    rng = np.random.default_rng(9)
    f_true = rng.normal(size=(B, N, N))
    b = np.stack([so.hough_project(f_true[s]) for s in range(B)]).astype(np.float32)
    plan = fbp.fbp_plan(N, K, M, B)
    img = torch.zeros(plan.img_shape, device="cuda")
    fbp.fbp_sirt(plan, torch.from_numpy(b).cuda(), img, iters, 1.2)
    assert fbp.fbp_last_device_error(plan) == 0
    got = img.cpu().numpy()
    for s in range(B):
        want = so.sirt(b[s].astype(np.float64), N, iters, 1.2)
        assert np.abs(got[s] - want).max() <= 1e-5 * np.abs(want).max()


@pytest.mark.parametrize("N", [16, 64])
def test_hough_data_and_radon_match_oracle_and_in_bounds(torch, N):
    import oracle.radon as orad
    import oracle.sirt as so
    K, M = phantoms.geometry_for(N)
    rng = np.random.default_rng(N + 3)
    sino = rng.normal(size=(2, K, M)).astype(np.float32)
    img = rng.random(size=(2, N, N)).astype(np.float32)
    plan = fbp.fbp_plan(N, K, M, 2)
    lin = torch.full(plan.lin_shape, float("nan"), device="cuda")
    fbp.fbp_hough_data(plan, torch.from_numpy(sino).cuda(), lin)
    rs = torch.full(plan.sino_shape, float("nan"), device="cuda")
    fbp.fbp_radon(plan, torch.from_numpy(img).cuda(), rs)
    assert fbp.fbp_last_device_error(plan) == 0
    got_lin, got_rs = lin.cpu().numpy(), rs.cpu().numpy()
    for s in range(2):
        want = so.hough_data(sino[s].astype(np.float64), N)
        assert np.abs(got_lin[s] - want).max() <= 1e-6 * np.abs(want).max()
        want = orad.fast_radon(img[s].astype(np.float64), K, M)
        assert np.abs(got_rs[s] - want).max() <= 1e-5 * np.abs(want).max()


def corrector_run(torch, flat, x, gy=None):
    B, N = x.shape[0], x.shape[-1]
    params = torch.tensor(flat, device="cuda")
    xd = torch.tensor(x.astype(np.float32), device="cuda")
    y = torch.full_like(xd, float("nan"))
    ws = torch.empty(fbp.fbp_cnn_workspace_bytes(N, B, True), dtype=torch.uint8, device="cuda")
    fbp.fbp_cnn_forward(params, xd, y, ws, train=True)
    g = None
    if gy is not None:
        g = torch.full_like(params, float("nan"))
        fbp.fbp_cnn_backward(params, xd, torch.tensor(gy.astype(np.float32), device="cuda"), g, ws)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64), (None if g is None else g.cpu().numpy().astype(np.float64))


@pytest.mark.parametrize("N,B", [(16, 3), (64, 2)])
def test_corrector_bit_exact_and_in_bounds(torch, N, B):
    # integer-valued networks (tests/cnn_inputs.py): forward and every parameter gradient
    # equal the oracle's bit for bit, with every index and bulk-copy range checked
    from cnn_inputs import flatten, int_images, int_params
    from oracle import cnn as ocnn
    rng = np.random.default_rng(200 + N)
    ps = int_params(7)
    x = int_images(rng, (B, N, N), 0.7)
    gy = int_images(rng, (B, N, N), 0.5)
    y, g = corrector_run(torch, flatten(ps), x, gy)
    assert fbp.fbp_cnn_last_error() == 0
    want_g = np.zeros(g.size)
    for b in range(B):
        yb, cache = ocnn.forward(ps, x[b], "bf16")
        assert np.array_equal(y[b], yb), f"N={N} image {b}: forward differs"
        grads, _ = ocnn.backward(ps, cache, gy[b], "bf16")
        want_g += flatten(grads).astype(np.float64)
    assert np.array_equal(g, want_g)


def test_corrector_failed_check_sets_its_status_word(torch):
    # the hook makes the last layer check its image accesses against one image: the second
    # image's loads and stores fail the check and are skipped, the first is unaffected
    from cnn_inputs import flatten, int_images, int_params
    from oracle import cnn as ocnn
    N, B = 16, 2
    rng = np.random.default_rng(5)
    ps = int_params(7)
    x = int_images(rng, (B, N, N), 0.7)
    fbp.fbp_check_cnn_image_limit(1)
    try:
        y, _ = corrector_run(torch, flatten(ps), x)
    finally:
        fbp.fbp_check_cnn_image_limit(0)
    assert fbp.fbp_cnn_last_error() == FBP_ERR_INTERNAL
    assert fbp.fbp_cnn_last_error() == 0                   # the read cleared it
    assert np.array_equal(y[0], ocnn.forward(ps, x[0], "bf16")[0])
    assert np.isnan(y[1]).all()                            # no output written
    y, _ = corrector_run(torch, flatten(ps), x)            # the hook is off again
    assert fbp.fbp_cnn_last_error() == 0
    assert np.array_equal(y[1], ocnn.forward(ps, x[1], "bf16")[0])


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
