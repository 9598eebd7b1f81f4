"""The learned corrector's kernels against the oracle CNN, and a training run that shows
the corrector moving fast reconstructions towards direct-FBP ones.

Two kinds of parity:
* Integer-valued networks (tests/cnn_inputs.py): every stored activation and gradient is an
  integer of magnitude <= 256 (exact in bfloat16) and every sum stays below 2^24 (exact in
  float32 in any order), so the output and every parameter gradient must equal the oracle's
  bit for bit.  The size (N = 256, 4 images: far more output tiles than the persistent
  convolution kernel has CTAs) makes every CTA run several iterations of its tile loop.
* Random networks: each output is compared, element by element, with the oracle evaluated
  at the kernels' storage precision (bfloat16 hidden weights, activations and gradients,
  oracle.cnn storage="bf16").  What remains is float32 accumulation and the bfloat16
  rounding decisions it can move: a moved decision changes one stored value by one
  bfloat16 unit, at most 2^-7 of it; to first order through the five stored layers the
  output moves by at most 5 * 2^-7 * A(p), A the same network run on |x| with |weights|
  and |biases| (an upper bound on every stored value's contribution).  The weight
  gradients get the same first-order bound with A replaced by sum_p |dL/dz| |input|.  In
  relative L2 the output stays within 2e-3 of the bfloat16 oracle; the weight gradients,
  sums of many products whose stored factors each carry such moved decisions from up to
  four layers below, within 2^-6.  Against the plain float64 network (no bfloat16 stores)
  the output stays within 3e-2 in relative L2.  The gradients are not compared with it: the
  first layer's gradients sum values that passed four bfloat16 stores, which alone moves
  them by 9% (weights) to 15% (biases) at N = 128 -- a property of the storage precision,
  which the bfloat16 oracle reproduces.
"""
import numpy as np
import pytest

import phantoms
from cnn_inputs import abs_gradient_bound, flatten, int_images, int_params, unflatten
from oracle import cnn as ocnn

pytestmark = pytest.mark.gpu

U7 = 2.0 ** -7        # one bfloat16 unit relative to the value, at most


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    return t


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def smooth_images(rng, B, N):
    x = rng.normal(size=(B, N + 4, N + 4))
    return (x[:, :-4, :-4] + x[:, 2:-2, 2:-2] + x[:, 4:, 4:]) / 3.0


def run_gpu(fbp, torch, flat, x, gy=None):
    """Forward (and backward with dL/dy = gy) through the C ABI; returns host arrays."""
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
    assert fbp.fbp_cnn_last_error() == 0
    return y.cpu().numpy().astype(np.float64), (None if g is None else g.cpu().numpy().astype(np.float64))


def test_integer_network_bit_exact_over_many_tiles(fbp, torch):
    N, B = 256, 4
    rng = np.random.default_rng(11)
    ps = int_params(3)
    x = int_images(rng, (B, N, N), 0.6)
    gy = int_images(rng, (B, N, N), 0.5)
    y, g = run_gpu(fbp, torch, flatten(ps), x, gy)
    want_g = np.zeros(g.size)
    bound = np.zeros(g.size)
    for b in range(B):
        yb, cache = ocnn.forward(ps, x[b], "bf16")
        # preconditions of exactness: integer stored values of magnitude <= 256
        for h in cache[1:]:
            assert np.array_equal(h, np.round(h)) and np.abs(h).max() <= 256
        assert np.array_equal(y[b], yb), f"image {b}: forward differs"
        grads, _ = ocnn.backward(ps, cache, gy[b], "bf16")
        want_g += flatten(grads).astype(np.float64)
        bound += flatten(abs_gradient_bound(ocnn, ps, cache, gy[b])).astype(np.float64)
    assert bound.max() < 2.0 ** 24                      # every partial sum exact in float32
    bad = np.flatnonzero(g != want_g)
    assert bad.size == 0, f"{bad.size} parameter gradients differ, first at {bad[:8]}"


@pytest.mark.parametrize("N,B", [(16, 3), (32, 1), (64, 2)])
def test_integer_network_bit_exact_smallest_sizes(fbp, torch, N, B):
    """The smallest images: 2 to 17 tensor-core tiles per image, first-layer rows of 4 to 16
    threads, pad records at both ends of every row handled by the same threads."""
    rng = np.random.default_rng(100 + N)
    ps = int_params(5)
    x = int_images(rng, (B, N, N), 0.7)
    gy = int_images(rng, (B, N, N), 0.5)
    y, g = run_gpu(fbp, torch, flatten(ps), x, gy)
    want_g = np.zeros(g.size)
    for b in range(B):
        yb, cache = ocnn.forward(ps, x[b], "bf16")
        assert np.array_equal(y[b], yb), f"N={N} image {b}: forward differs"
        grads, _ = ocnn.backward(ps, cache, gy[b], "bf16")
        want_g += flatten(grads).astype(np.float64)
    assert np.array_equal(g, want_g)


def test_last_layer_weight_split_is_exact(fbp, torch):
    """The 32 -> 1 layer multiplies its float32 weights on the tensor cores as three bfloat16
    parts (hi + mid + lo).  Hidden layers with zero weights and bias 1 make every hidden
    activation 1 inside the image; two last-layer weights need all three parts
    (1 + 2^-9 + 2^-18: hi = 1, mid = 2^-9, lo = 2^-18), and every partial sum of the output
    stays within 22 significant bits, so the output must equal the float64 network exactly.
    Dropping a part, or rounding a weight to bfloat16, moves it."""
    N, B = 64, 2
    ps = [(np.zeros((32, 1, 3, 3)), np.ones(32))]
    ps += [(np.zeros((32, 32, 3, 3)), np.ones(32)) for _ in range(4)]
    w6 = np.zeros((1, 32, 3, 3))
    w6[0, 0, 1, 1] = 1.0 + 2.0 ** -9 + 2.0 ** -18
    w6[0, 5, 0, 2] = 2.0 ** -3 + 2.0 ** -12 + 2.0 ** -20
    ps.append((w6, np.array([0.25])))
    rng = np.random.default_rng(7)
    x = rng.integers(-3, 4, size=(B, N, N)).astype(np.float64)
    y, _ = run_gpu(fbp, torch, flatten(ps), x)
    for b in range(B):
        want, _ = ocnn.forward(ps, x[b], "f64")
        assert np.array_equal(y[b], want), float(np.abs(y[b] - want).max())
    # the float32 weights are what the library was given
    assert float(np.float32(w6[0, 0, 1, 1])) == w6[0, 0, 1, 1]


def random_params(seed, rng):
    from paper_2007_06289_gb300 import corrector
    flat = corrector.init_params(seed=seed, scale=2.0)
    flat[-289:] *= 10.0                              # a last layer of normal size
    flat[:] += rng.normal(0, 0.02, flat.size).astype(np.float32)   # nonzero biases
    return flat


def test_forward_matches_oracle_elementwise(fbp, torch):
    rng = np.random.default_rng(0)
    B, N = 2, 128
    flat = random_params(1, rng)
    x = smooth_images(rng, B, N).astype(np.float32).astype(np.float64)
    y, _ = run_gpu(fbp, torch, flat, x)
    ps = unflatten(flat)
    aps = [(np.abs(w), np.abs(bb)) for w, bb in ps]
    for b in range(B):
        want16, _ = ocnn.forward(ps, x[b], "bf16")
        want64, _ = ocnn.forward(ps, x[b], "f64")
        A = ocnn.forward(aps, np.abs(x[b]))[0] - np.abs(x[b])
        err = np.abs(y[b] - want16)
        assert np.all(err <= 5 * U7 * A + 1e-6 * np.abs(want16).max()), float((err / A).max())
        assert rel(y[b] - x[b], want16 - x[b]) <= 2e-3
        assert rel(y[b] - x[b], want64 - x[b]) <= 3e-2


def test_gradients_match_oracle_elementwise(fbp, torch):
    rng = np.random.default_rng(1)
    B, N = 2, 128
    flat = random_params(2, rng)
    x = smooth_images(rng, B, N).astype(np.float32).astype(np.float64)
    gy = (rng.normal(size=(B, N, N)) / (B * N * N)).astype(np.float32).astype(np.float64)
    _, g = run_gpu(fbp, torch, flat, x, gy)
    ps = unflatten(flat)
    want16 = np.zeros(g.size)
    bound = np.zeros(g.size)
    for b in range(B):
        _, c16 = ocnn.forward(ps, x[b], "bf16")
        g16, _ = ocnn.backward(ps, c16, gy[b], "bf16")
        want16 += flatten(g16)
        bound += flatten(abs_gradient_bound(ocnn, ps, c16, gy[b]))
    err = np.abs(g - want16)
    assert np.all(err <= 5 * U7 * bound + 1e-6 * np.abs(want16).max())
    off = 0
    for k, (w, bb) in enumerate(ps):
        n = w.size + bb.size
        sl_w, sl_b = slice(off, off + w.size), slice(off + w.size, off + n)
        assert rel(g[sl_w], want16[sl_w]) <= 2.0 ** -6, k
        assert rel(g[sl_b], want16[sl_b]) <= 2.0 ** -6, k
        off += n


def window_forward(ps, x, y0, x0, storage):
    """The network's output at pixel (y0, x0) of the N x N image x, from the 13 x 13 window
    of inputs around it (six 3 x 3 layers: an output depends on inputs within 6 pixels).  The
    oracle's layers run on the window, each layer's values zeroed off the image as the
    network's zero padding does; the window's own edge only corrupts values that no longer
    reach the centre."""
    N, R = x.shape[-1], 6
    ys, xs = np.arange(y0 - R, y0 + R + 1), np.arange(x0 - R, x0 + R + 1)
    inside = ((ys[:, None] >= 0) & (ys[:, None] < N) & (xs[None, :] >= 0) & (xs[None, :] < N))
    win = np.where(inside, x[np.clip(ys, 0, N - 1)][:, np.clip(xs, 0, N - 1)], 0.0)
    stored = ocnn._stored(ps, storage)
    h = win[None]
    for k, (w, b) in enumerate(stored):
        z = ocnn.conv3x3(h, w, b)
        if k < len(stored) - 1:
            h = np.maximum(z, 0.0)
            if storage == "bf16":
                h = ocnn.bf16(h)
            h = h * inside
        else:
            h = z
    return win[R, R] + h[0, R, R]


def sample_pixels(rng, N, n):
    """Corners, the middle of every edge and random pixels (row ends straddle tiles)."""
    fixed = [(0, 0), (0, N - 1), (N - 1, 0), (N - 1, N - 1), (0, N // 2), (N - 1, N // 2),
             (N // 2, 0), (N // 2, N - 1), (1, 1), (N - 2, N - 2)]
    rand = [tuple(p) for p in rng.integers(0, N, size=(n - len(fixed), 2))]
    return fixed + rand


def test_full_size_sampled_pixels_match_oracle(fbp, torch):
    """N = 2048 (the inference size of the benchmark), two images: an integer network bit for
    bit and a random network within the first-order bfloat16 bound, at sampled pixels
    (corners, edges, interior) evaluated one by one by the oracle on their input windows."""
    N, B = 2048, 2
    rng = np.random.default_rng(2048)
    pix = sample_pixels(rng, N, 40)
    # integer network: exact
    ps = int_params(9)
    x = int_images(rng, (B, N, N), 0.6)
    y, _ = run_gpu(fbp, torch, flatten(ps), x)
    for b in range(B):
        for (py, px) in pix:
            want = window_forward(ps, x[b], py, px, "bf16")
            assert y[b, py, px] == want, (b, py, px, y[b, py, px], want)
    # random network: within 5 * 2^-7 * A of the bfloat16-storage oracle
    flat = random_params(3, rng)
    x = smooth_images(rng, B, N).astype(np.float32).astype(np.float64)
    y, _ = run_gpu(fbp, torch, flat, x)
    ps = unflatten(flat)
    aps = [(np.abs(w), np.abs(bb)) for w, bb in ps]
    for b in range(B):
        for (py, px) in pix:
            want = window_forward(ps, x[b], py, px, "bf16")
            A = window_forward(aps, np.abs(x[b]), py, px, "f64") - abs(x[b, py, px])
            assert abs(y[b, py, px] - want) <= 5 * U7 * A + 1e-6 * abs(want), (b, py, px)


def test_training_reduces_the_error_to_direct_fbp(fbp, torch):
    from paper_2007_06289_gb300 import corrector
    N, S = 64, 16
    K, M = phantoms.geometry_for(N)
    sino = phantoms.phantom_stack_torch(N, S, 500, "cuda", noise_i0=1e5)
    fast = torch.empty(S, N, N, device="cuda")
    direct = torch.empty(S, N, N, device="cuda")
    fbp.fbp_reconstruct(fbp.fbp_plan(N, K, M, S), sino, fast)
    fbp.fbp_direct_reconstruct(fbp.fbp_plan(N, K, M, S), sino, direct)
    torch.cuda.synchronize()
    train, test = slice(0, 12), slice(12, 16)
    params, losses = corrector.train(fast[train], direct[train], steps=400, batch=4, lr=2e-3)
    before = float(torch.sqrt(torch.mean((fast[test] - direct[test]) ** 2)))
    after = float(torch.sqrt(torch.mean((corrector.infer(params, fast[test].contiguous())
                                         - direct[test]) ** 2)))
    assert np.mean(losses[-20:]) < np.mean(losses[:20])
    assert after < 0.9 * before, (before, after)
