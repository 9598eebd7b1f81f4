"""Pins of the oracle CNN corrector: the convolution against scipy's 2-D correlation, every
hand-written gradient against float64 finite differences, and the identity start."""
import numpy as np
import pytest

from oracle import cnn


def test_conv_is_a_sum_of_2d_correlations():
    from scipy.signal import correlate2d
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 7, 9))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    got = cnn.conv3x3(x, w, b)
    for o in range(4):
        want = b[o] + sum(correlate2d(x[i], w[o, i], mode="same", boundary="fill")
                          for i in range(3))
        np.testing.assert_allclose(got[o], want, rtol=0, atol=1e-12)


def fd(f, x, d, h=1e-6):
    return (f(x + h * d) - f(x - h * d)) / (2 * h)


def test_conv_gradients_by_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 5, 6))
    w = rng.normal(size=(3, 2, 3, 3))
    b = rng.normal(size=3)
    u = rng.normal(size=(3, 5, 6))            # L = <u, conv(x)>
    gx, gw, gb = cnn.conv3x3_backward(x, w, u)
    for _ in range(8):
        dx = rng.normal(size=x.shape)
        dw = rng.normal(size=w.shape)
        db = rng.normal(size=b.shape)
        assert abs(fd(lambda t: np.sum(u * cnn.conv3x3(t, w, b)), x, dx) - np.sum(gx * dx)) < 1e-7
        assert abs(fd(lambda t: np.sum(u * cnn.conv3x3(x, t, b)), w, dw) - np.sum(gw * dw)) < 1e-7
        assert abs(fd(lambda t: np.sum(u * cnn.conv3x3(x, w, t)), b, db) - np.sum(gb * db)) < 1e-7


def test_network_gradients_by_finite_differences():
    rng = np.random.default_rng(2)
    params = cnn.init_params(channels=4, layers=6, seed=3, scale=3.0)
    # biases nonzero so that ReLUs switch inside the net
    params = [(w, rng.normal(0, 0.1, size=b.shape)) for w, b in params]
    x = rng.normal(size=(6, 7))
    t = rng.normal(size=(6, 7))
    loss, grads, gx = cnn.loss_and_grads(params, x, t)

    def total(ps, xx):
        y, _ = cnn.forward(ps, xx)
        return float(np.mean((y - t) ** 2))

    for k in (0, 2, 5):
        w, b = params[k]
        for _ in range(4):
            dw = rng.normal(size=w.shape)
            f = lambda s: total([(w + s * dw if j == k else pw, pb) for j, (pw, pb) in enumerate(params)], x)
            num = (f(1e-6) - f(-1e-6)) / 2e-6
            assert abs(num - np.sum(grads[k][0] * dw)) <= 1e-6 * max(1.0, abs(num))
            db = rng.normal(size=b.shape)
            f = lambda s: total([(pw, b + s * db if j == k else pb) for j, (pw, pb) in enumerate(params)], x)
            num = (f(1e-6) - f(-1e-6)) / 2e-6
            assert abs(num - np.sum(grads[k][1] * db)) <= 1e-6 * max(1.0, abs(num))
    for _ in range(4):
        d = rng.normal(size=x.shape)
        num = (total(params, x + 1e-6 * d) - total(params, x - 1e-6 * d)) / 2e-6
        assert abs(num - np.sum(gx * d)) <= 1e-6 * max(1.0, abs(num))


def test_zero_last_layer_is_the_identity():
    params = cnn.init_params(channels=4, seed=1)
    params[-1] = (np.zeros_like(params[-1][0]), np.zeros_like(params[-1][1]))
    x = np.random.default_rng(3).normal(size=(5, 5))
    y, _ = cnn.forward(params, x)
    np.testing.assert_array_equal(y, x)


def test_bf16_rounding_matches_torch_and_ties_to_even():
    import torch
    rng = np.random.default_rng(4)
    x = rng.normal(size=2000) * 10.0 ** rng.integers(-8, 8, 2000)
    x = np.concatenate([x, [0.0, -0.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 255.0, 257.0]])
    want = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(cnn.bf16(x), want)
    assert cnn.bf16(1 + 2 ** -8) == 1.0                  # tie -> even mantissa
    assert cnn.bf16(1 + 3 * 2 ** -8) == 1 + 2 ** -6      # tie -> even mantissa
    assert cnn.bf16(255.0) == 255.0 and cnn.bf16(257.0) == 256.0


def test_bf16_storage_is_exact_on_integer_networks():
    from cnn_inputs import int_images, int_params
    rng = np.random.default_rng(5)
    ps = int_params(3)
    x = int_images(rng, (24, 24), 0.6)
    gy = int_images(rng, (24, 24), 0.5)
    y16, c16 = cnn.forward(ps, x, "bf16")
    y64, c64 = cnn.forward(ps, x, "f64")
    np.testing.assert_array_equal(y16, y64)
    g16, gx16 = cnn.backward(ps, c16, gy, "bf16")
    g64, gx64 = cnn.backward(ps, c64, gy, "f64")
    for (a, b), (c, d) in zip(g16, g64):
        np.testing.assert_array_equal(a, c)
        np.testing.assert_array_equal(b, d)
    np.testing.assert_array_equal(gx16, gx64)
    assert max(np.abs(h).max() for h in c16[1:]) <= 256


def test_bf16_storage_rounds_the_stored_values():
    rng = np.random.default_rng(6)
    ps = cnn.init_params(channels=8, seed=2, scale=2.0)
    ps = [(w, rng.normal(0, 0.1, size=b.shape)) for w, b in ps]
    x = rng.normal(size=(10, 11))
    y16, c16 = cnn.forward(ps, x, "bf16")
    y64, _ = cnn.forward(ps, x, "f64")
    for h in c16[1:]:                                   # stored hidden activations
        np.testing.assert_array_equal(cnn.bf16(h), h)
    assert 0 < np.abs(y16 - y64).max() <= 0.05 * np.abs(y64 - x).max()
    gy = rng.normal(size=x.shape)
    g16, _ = cnn.backward(ps, c16, gy, "bf16")
    # a hidden layer's weight gradient is a sum of products of stored (bfloat16) values:
    # planting float64 gradients in the bfloat16 pass changes it
    g64, _ = cnn.backward(ps, c16, gy, "f64")
    assert not np.array_equal(g16[2][0], g64[2][0])
    assert np.abs(g16[2][0] - g64[2][0]).max() <= 0.05 * np.abs(g64[2][0]).max()
