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
