"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (derivations in the design notes):
* recursive filter: max |gpu - oracle| <= 1e-5 * max |oracle| (float32 parallel form;
  measured float32 error ~2e-6 of the peak);
* resampling: max |gpu - oracle| <= 2e-6 * max|p~| * max(w) (float32 bilinear weights of
  float32 samples, positions carried in 32.32 fixed point);
* Hough back projection: bit for bit against the float32 stage recursion, and exactly equal
  to float64 brute-force pattern sums on integer-valued inputs;
* whole pipeline: max |gpu - oracle| <= 1e-5 * (max - min) of the image (float64 oracle);
* direct comparator: max |gpu - oracle| <= 2e-4 * (max - min) (float32 detector positions).
"""
import ctypes

import numpy as np
import pytest

import oracle
import phantoms

pytestmark = pytest.mark.gpu

TOL_IIR = 1e-5
TOL_PIPE = 1e-5
TOL_DIRECT = 2e-4


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    return t


def coeffs(table, N, order=3):
    for e in table["entries"]:
        if e["N"] == N and e["order"] == order:
            return list(e["b"]), list(e["a"])
    raise KeyError((N, order))


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def gpu_filter(fbp, torch, sino, N, co):
    B, K, M = sino.shape
    plan = fbp.fbp_plan(N, K, M, B, co)
    x = dev(torch, sino)
    y = torch.empty_like(x)
    fbp.fbp_filter_iir(plan, x, y)
    torch.cuda.synchronize()
    return host(y)


# ------------------------------------------------------------------ recursive filter
@pytest.mark.parametrize("N,order,noise", [(256, 2, False), (256, 3, False), (256, 4, True),
                                           (256, 5, False), (256, 6, True), (2048, 3, True),
                                           (2048, 6, False), (16, 3, False), (2, 3, False)])
def test_iir_filter_matches_oracle(fbp, torch, coeff_table, N, order, noise):
    K, M = phantoms.geometry_for(N)
    K = min(K, 96)
    ell = phantoms.random_ellipses(N + order)
    s = phantoms.ellipse_sinogram(ell, N, K, M, 1e5 if noise else None, 5)[None].astype(np.float32)
    co = coeffs(coeff_table, N, order)
    got = gpu_filter(fbp, torch, s, N, co)[0]
    want = oracle.iir_filter(s[0].astype(np.float64), *co)
    assert np.abs(got - want).max() <= TOL_IIR * np.abs(want).max()


@pytest.mark.parametrize("M", [2, 3, 31, 32, 33, 95, 725, 1000, 2897, 5793])
def test_iir_filter_ragged_rows(fbp, torch, coeff_table, M):
    rng = np.random.default_rng(M)
    s = rng.normal(size=(2, 5, M)).astype(np.float32)
    co = coeffs(coeff_table, 1024, 4)
    got = gpu_filter(fbp, torch, s, 16, co)
    want = oracle.iir_filter(s.astype(np.float64), *co)
    assert np.abs(got - want).max() <= TOL_IIR * np.abs(want).max()


def test_iir_filter_pure_fir_and_complex_poles(fbp, torch):
    rng = np.random.default_rng(3)
    s = rng.normal(size=(1, 7, 300)).astype(np.float32)
    # 2897 samples per row: lanes of 23 samples (the unrolled kernel variant)
    s2 = rng.normal(size=(1, 5, 2897)).astype(np.float32)
    for co in ([0.1, 0.2, -0.3], list(np.real(np.poly([0.6 + 0.5j, 0.6 - 0.5j, 0.3]))[1:])), \
              ([0.2, -0.1, 0.05], list(np.real(np.poly([0.9 + 0.2j, 0.9 - 0.2j, -0.4, 0.5]))[1:])):
        got = gpu_filter(fbp, torch, s2, 2048, co)
        want = oracle.iir_filter(s2.astype(np.float64), *co)
        assert np.abs(got - want).max() <= TOL_IIR * np.abs(want).max()
    for co in (([0.25, -0.5, 0.25], []),                                   # no feedback
               ([0.1, 0.2, -0.3], list(np.real(np.poly([0.6 + 0.5j, 0.6 - 0.5j, 0.3]))[1:])),
               ([0.3, -0.1, 0.05, 0.02, -0.01], [-0.5, 0.06])):           # direct taps
        got = gpu_filter(fbp, torch, s, 16, co)
        want = oracle.iir_filter(s.astype(np.float64), *co)
        assert np.abs(got - want).max() <= TOL_IIR * np.abs(want).max()


def test_iir_filter_in_place(fbp, torch, coeff_table):
    rng = np.random.default_rng(1)
    s = rng.normal(size=(3, 40, 363)).astype(np.float32)
    plan = fbp.fbp_plan(256, 40, 363, 3, coeffs(coeff_table, 256))
    x = dev(torch, s)
    y = torch.empty_like(x)
    fbp.fbp_filter_iir(plan, x, y)
    fbp.fbp_filter_iir(plan, x, x)
    torch.cuda.synchronize()
    assert torch.equal(x, y)


# ------------------------------------------------------------------ resampling
@pytest.mark.parametrize("N", [2, 8, 64, 256])
def test_resample_matches_oracle(fbp, torch, N):
    K, M = phantoms.geometry_for(N)
    rng = np.random.default_rng(N)
    pt = rng.normal(size=(2, K, M)).astype(np.float32)
    plan = fbp.fbp_plan(N, K, M, 2)
    lin = torch.empty(plan.lin_shape, device="cuda")
    fbp.fbp_resample_st(plan, dev(torch, pt), lin)
    torch.cuda.synchronize()
    got = host(lin)
    wmax = oracle.row_weights(N).max()
    for b in range(2):
        want = oracle.linogram(pt[b].astype(np.float64), N)
        assert np.abs(got[b] - want).max() <= 2e-6 * np.abs(pt[b]).max() * wmax


# ------------------------------------------------------------------ Hough back projection
def gpu_fht(fbp, torch, lin, N, fuse_k=0):
    B = lin.shape[0]
    K, M = phantoms.geometry_for(N)
    plan = fbp.fbp_plan(N, K, M, B, None, fuse_k)
    img = torch.empty(plan.img_shape, device="cuda")
    fbp.fbp_fht_backproject(plan, dev(torch, lin), img)
    torch.cuda.synchronize()
    return host(img)


@pytest.mark.parametrize("N,fuse_k", [(2, 0), (4, 0), (8, 0), (16, 0), (32, 0), (64, 0),
                                      (128, 0), (256, 0), (256, 2), (256, 3), (256, 5),
                                      (256, 6), (512, 0), (512, 6), (1024, 4)])
def test_fht_bit_exact(fbp, torch, N, fuse_k):
    rng = np.random.default_rng(N + fuse_k)
    lin = rng.normal(size=(2, 4, N, 2 * N)).astype(np.float32)
    got = gpu_fht(fbp, torch, lin, N, fuse_k)
    for b in range(2):
        want = oracle.fht_backproject(lin[b])
        np.testing.assert_array_equal(got[b], want)


def test_fht_bit_exact_full_size_2048(fbp, torch):
    N = 2048
    rng = np.random.default_rng(2048)
    lin = rng.normal(size=(1, 4, N, 2 * N)).astype(np.float32)
    got = gpu_fht(fbp, torch, lin, N)
    np.testing.assert_array_equal(got[0], oracle.fht_backproject(lin[0]))


@pytest.mark.parametrize("N", [2048, 4096])
def test_fht_integer_inputs_exact_on_sampled_pixels(fbp, torch, N):
    # |values| <= 2^10 and 4N terms keep every partial sum an exact float32 integer, so the
    # GPU must equal float64 brute-force pattern sums exactly.
    rng = np.random.default_rng(N)
    lin = rng.integers(-1024, 1025, size=(1, 4, N, 2 * N)).astype(np.float32)
    got = gpu_fht(fbp, torch, lin, N)[0]
    n = N.bit_length() - 1
    L = lin[0].astype(np.float64)
    rows = np.arange(N)
    for y, x in zip(rng.integers(0, N, 40), rng.integers(0, N, 40)):
        dy, dx = oracle.dyadic_pattern(n, int(y)), oracle.dyadic_pattern(n, int(x))
        v = (L[0, rows, x + dy].sum() + L[1, rows, N - 1 - x + dy].sum()) + \
            (L[2, rows, y + dx].sum() + L[3, rows, N - 1 - y + dx].sum())
        assert got[y, x] == v


# ------------------------------------------------------------------ whole pipeline
def test_reconstruct_equals_composition_bitwise(fbp, torch, coeff_table):
    N = 256
    K, M = phantoms.geometry_for(N)
    s = phantoms.phantom_stack(N, 3, 300, 1e5)
    plan = fbp.fbp_plan(N, K, M, 3, coeffs(coeff_table, N, 4))
    x = dev(torch, s)
    filt = torch.empty_like(x)
    lin = torch.empty(plan.lin_shape, device="cuda")
    a = torch.empty(plan.img_shape, device="cuda")
    b = torch.empty(plan.img_shape, device="cuda")
    fbp.fbp_filter_iir(plan, x, filt)
    fbp.fbp_resample_st(plan, filt, lin)
    fbp.fbp_fht_backproject(plan, lin, a)
    fbp.fbp_reconstruct(plan, x, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("order", [3, 5])
def test_pipeline_matches_fp64_oracle_n256(fbp, torch, coeff_table, order):
    # The single-slice workload: N = 256, K = 384, M = 363, ten-ellipse phantom, seed 2020.
    N = 256
    K, M = phantoms.geometry_for(N)
    s = phantoms.ellipse_sinogram(phantoms.random_ellipses(2020), N, K, M).astype(np.float32)
    co = coeffs(coeff_table, N, order)
    plan = fbp.fbp_plan(N, K, M, 1, co)
    img = torch.empty(plan.img_shape, device="cuda")
    fbp.fbp_reconstruct(plan, dev(torch, s[None]), img)
    torch.cuda.synchronize()
    want = oracle.fast_fbp(s.astype(np.float64), N, *co)
    got = host(img)[0]
    assert np.abs(got - want).max() <= TOL_PIPE * (want.max() - want.min())


def test_pipeline_matches_fp64_oracle_at_full_size(fbp, torch, coeff_table):
    # The benchmark's launch configuration: N = 2048, K = 3072, M = 2897, 64 noisy slices
    # in one call; sampled pixels of two slices against the float64 oracle.
    N, B = 2048, 64
    K, M = phantoms.geometry_for(N)
    sino = phantoms.phantom_stack_torch(N, B, 2021, "cuda", noise_i0=1e5)
    co = coeffs(coeff_table, N, 3)
    plan = fbp.fbp_plan(N, K, M, B, co)
    img = torch.empty(plan.img_shape, device="cuda")
    fbp.fbp_reconstruct(plan, sino, img)
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    for sl in (0, B - 1):
        s = host(sino[sl]).astype(np.float64)
        got = host(img[sl])
        ys, xs = rng.integers(0, N, 24), rng.integers(0, N, 24)
        ys[:4] = [0, N - 1, 0, N - 1]
        xs[:4] = [0, 0, N - 1, N - 1]
        want = oracle.fast_fbp_pixels(s, N, *co, ys, xs)
        assert np.abs(got[ys, xs] - want).max() <= TOL_PIPE * (got.max() - got.min())


def test_pipeline_matches_fp64_oracle_at_largest_size(fbp, torch, coeff_table):
    # N = 4096 (K = 6144, M = 5793), the largest supported size: two slices, sampled pixels
    N, B = 4096, 2
    K, M = phantoms.geometry_for(N)
    sino = phantoms.phantom_stack_torch(N, B, 4096, "cuda", noise_i0=1e5)
    co = coeffs(coeff_table, N, 3)
    plan = fbp.fbp_plan(N, K, M, B, co)
    img = torch.empty(plan.img_shape, device="cuda")
    fbp.fbp_reconstruct(plan, sino, img)
    torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    s = host(sino[1]).astype(np.float64)
    got = host(img[1])
    ys, xs = rng.integers(0, N, 12), rng.integers(0, N, 12)
    ys[:2] = [0, N - 1]
    xs[:2] = [N - 1, 0]
    want = oracle.fast_fbp_pixels(s, N, *co, ys, xs)
    assert np.abs(got[ys, xs] - want).max() <= TOL_PIPE * (got.max() - got.min())


def test_chunked_batch_and_host_api(fbp, torch, coeff_table):
    # Chunks of 4 slices: a batch of 5 ends with a ragged chunk (and the host path, which
    # stages 2 slices per copy, with a ragged stage).
    N, B = 1024, 5
    K, M = phantoms.geometry_for(N)
    sino = phantoms.phantom_stack_torch(N, B, 40, "cuda", noise_i0=1e5)
    co = coeffs(coeff_table, N, 3)
    plan = fbp.fbp_plan(N, K, M, B, co)
    assert plan.chunk == B                          # default: the whole batch of 5
    fbp.fbp_set_chunk(plan, 4)
    assert plan.chunk == 4
    img = torch.empty(plan.img_shape, device="cuda")
    fbp.fbp_reconstruct(plan, sino, img)
    single = fbp.fbp_plan(N, K, M, 1, co)
    one = torch.empty(single.img_shape, device="cuda")
    hs = sino.cpu().pin_memory()
    hi = torch.empty(plan.img_shape, pin_memory=True)
    fbp.fbp_reconstruct_host(plan, hs, hi)
    torch.cuda.synchronize()
    for b in range(B):
        fbp.fbp_reconstruct(single, sino[b:b + 1].contiguous(), one)
        torch.cuda.synchronize()
        assert torch.equal(one[0], img[b])
    assert torch.equal(hi, img.cpu())
    # every chunk size gives the same bits
    for chunk in (1, 2, 3, 5):
        p2 = fbp.fbp_plan(N, K, M, B, co)
        fbp.fbp_set_chunk(p2, chunk)
        assert p2.chunk == chunk
        img2 = torch.empty(plan.img_shape, device="cuda")
        fbp.fbp_reconstruct(p2, sino, img2)
        torch.cuda.synchronize()
        assert torch.equal(img2, img)
    with pytest.raises(fbp.FbpError):
        fbp.fbp_set_chunk(plan, 2)                  # the plan already has its workspace
    with pytest.raises(fbp.FbpError):
        fbp.fbp_set_chunk(fbp.fbp_plan(N, K, M, B, co), B + 1)


@pytest.mark.parametrize("window", ["shepp-logan", "hann"])
def test_windowed_filters_match_oracle(fbp, torch, window):
    # other FBP filters through the recursive fit: the GPU pipeline with those coefficients
    # against the float64 oracle with the same coefficients
    from paper_2007_06289_gb300 import iir_fit
    N = 256
    K, M = phantoms.geometry_for(N)
    b, a = iir_fit.window_coefficients(N, window)
    s = phantoms.phantom_stack(N, 1, 77, noise_i0=1e5)
    plan = fbp.fbp_plan(N, K, M, 1, (list(b), list(a)))
    img = torch.empty(plan.img_shape, device="cuda")
    fbp.fbp_reconstruct(plan, dev(torch, s), img)
    torch.cuda.synchronize()
    want = oracle.fast_fbp(s[0].astype(np.float64), N, b, a)
    assert np.abs(host(img)[0] - want).max() <= TOL_PIPE * (want.max() - want.min())


def test_linearity(fbp, torch, coeff_table):
    N = 128
    K, M = phantoms.geometry_for(N)
    s = phantoms.phantom_stack(N, 2, 11)
    plan = fbp.fbp_plan(N, K, M, 1, coeffs(coeff_table, N, 3))
    outs = []
    for arr in (s[0], s[1], 2.0 * s[0] - 0.5 * s[1]):
        img = torch.empty(plan.img_shape, device="cuda")
        fbp.fbp_reconstruct(plan, dev(torch, arr[None]), img)
        outs.append(host(img)[0].astype(np.float64))
    comb = 2.0 * outs[0] - 0.5 * outs[1]
    assert np.abs(outs[2] - comb).max() <= 1e-5 * (comb.max() - comb.min())


# ------------------------------------------------------------------ direct comparator
def test_direct_fbp_matches_oracle(fbp, torch):
    for N, sample in ((64, False), (1024, True)):
        K, M = phantoms.geometry_for(N)
        s = phantoms.ellipse_sinogram(phantoms.random_ellipses(N), N, K, M).astype(np.float32)
        plan = fbp.fbp_plan(N, K, M, 1)
        img = torch.empty(plan.img_shape, device="cuda")
        fbp.fbp_direct_reconstruct(plan, dev(torch, s[None]), img)
        torch.cuda.synchronize()
        got = host(img)[0]
        if not sample:
            want = oracle.direct_fbp(s.astype(np.float64), N)
            assert np.abs(got - want).max() <= TOL_DIRECT * (want.max() - want.min())
        else:
            rng = np.random.default_rng(0)
            ys, xs = rng.integers(0, N, 64), rng.integers(0, N, 64)
            want = oracle.direct_fbp_pixels(s.astype(np.float64), N, ys, xs)
            assert np.abs(got[ys, xs] - want).max() <= TOL_DIRECT * (got.max() - got.min())


def test_direct_fbp_partial_tile_sizes(fbp, torch):
    # sizes below and across the comparator's 32 x 32 pixel tile and 32-angle blocks
    for N, K, M in ((2, 3, 3), (16, 24, 23), (32, 37, 67), (64, 31, 129)):
        s = phantoms.ellipse_sinogram(phantoms.random_ellipses(N + 1), N, K, M).astype(np.float32)
        plan = fbp.fbp_plan(N, K, M, 1)
        img = torch.empty(plan.img_shape, device="cuda")
        fbp.fbp_direct_reconstruct(plan, dev(torch, s[None]), img)
        torch.cuda.synchronize()
        want = oracle.direct_fbp(s.astype(np.float64), N)
        assert np.abs(host(img)[0] - want).max() <= TOL_DIRECT * max(want.max() - want.min(), 1e-6)


def test_exact_fir_filter_matches_oracle(fbp, torch):
    # fbp_filter_fir: the exact ramp filter of Eq. 8 over whole rows (the comparator's filter).
    # A float32 sum of up to M terms with heavy cancellation: each output is bounded by
    # 2^-14 of the sum of its terms' magnitudes, sum_k |h(k)| |p(n-k)| (the recursive-sum
    # bound M 2^-24 of that sum is 2^-13.5 at M = 1449); a wrong tap or bin is off by a
    # whole term.
    from scipy.signal import fftconvolve
    for N in (64, 1024):
        K, M = phantoms.geometry_for(N)
        s = phantoms.ellipse_sinogram(phantoms.random_ellipses(N + 7), N, K, M, 1e5, 3).astype(np.float32)
        plan = fbp.fbp_plan(N, K, M, 1)
        out = torch.empty(plan.sino_shape, device="cuda")
        fbp.fbp_filter_fir(plan, dev(torch, s[None]), out)
        s64 = s.astype(np.float64)
        want = oracle.fir_ramp(s64)
        habs = np.abs(oracle.ramp_h(np.arange(-(M - 1), M)))
        mag = fftconvolve(np.abs(s64), habs[None, :], mode="same", axes=1)
        err = np.abs(host(out)[0] - want)
        assert np.all(err <= 2.0 ** -14 * mag), float((err / mag).max())


# ------------------------------------------------------------------ ABI behaviour on a GPU
def test_misaligned_and_workspace(fbp, torch):
    N = 64
    K, M = phantoms.geometry_for(N)
    plan = fbp.fbp_plan(N, K, M, 1)
    lib = fbp.load_library()
    buf = torch.zeros(K * M + 8, device="cuda")
    img = torch.empty(N * N + 8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    rc = lib.fbp_reconstruct(plan.handle, ctypes.c_void_p(buf.data_ptr() + 4),
                             ctypes.c_void_p(img.data_ptr()), ctypes.c_void_p(st))
    assert rc == 3
    ws = torch.empty(fbp.fbp_workspace_bytes(plan), dtype=torch.uint8, device="cuda")
    fbp.fbp_set_workspace(plan, ws)
    s = phantoms.ellipse_sinogram(phantoms.random_ellipses(1), N, K, M).astype(np.float32)
    a = torch.empty(plan.img_shape, device="cuda")
    fbp.fbp_reconstruct(plan, dev(torch, s[None]), a)
    other = fbp.fbp_plan(N, K, M, 1)
    b = torch.empty(plan.img_shape, device="cuda")
    fbp.fbp_reconstruct(other, dev(torch, s[None]), b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert fbp.fbp_last_device_error(plan) == 0
