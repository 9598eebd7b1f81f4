"""Pins of the oracle's algebraic reconstruction on the fast Hough operators (oracle.sirt).

* The two operators are transposes of each other (adjoint identity), and SIRT with them
  recovers the image that produced consistent data (it converges to it: a wrong weight, a
  sign or a non-transposed pair stops that).
* On noisy data the weighted residual never increases (0 < lambda < 2).
* Hough-space data: a constant sinogram gives c / sqrt(1 + sigma^2) wherever the line falls
  on the detector (closed form), and the closed-form sinogram of a disk gives what the
  projector makes of the rasterised disk (the path-length scale; a missing or inverted
  sqrt(1 + sigma^2) is off by up to a factor 2 on the steep lines).
"""
import numpy as np

import oracle.sirt as so
import phantoms
from oracle.geometry import quarter_r, slopes


def test_operators_are_transposes():
    N = 8
    rng = np.random.default_rng(0)
    f = rng.normal(size=(N, N))
    L = rng.normal(size=(4, N, 2 * N))
    lhs = float(np.sum(so.hough_project(f) * L))
    rhs = float(np.sum(f * so.back_project(L)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_sirt_converges_to_the_image_on_consistent_data():
    N = 8
    rng = np.random.default_rng(1)
    f_true = rng.normal(size=(N, N))
    b = so.hough_project(f_true)
    err = [np.linalg.norm(so.sirt(b, N, it, 1.0) - f_true) / np.linalg.norm(f_true)
           for it in (10, 100, 400)]
    assert err[0] > err[1] > err[2]
    assert err[2] < 1e-6


def test_sirt_weighted_residual_never_increases_on_noisy_data():
    N = 8
    rng = np.random.default_rng(2)
    b = so.hough_project(rng.normal(size=(N, N)))
    b = b + 0.1 * rng.normal(size=b.shape) * (b != 0)
    rinv, _ = so.sirt_weights(N)
    f = np.zeros((N, N))
    prev = np.inf
    for _ in range(30):
        f = so.sirt(b, N, 1, 1.5, f0=f)
        r = b - so.hough_project(f)
        cur = float(np.sum(rinv * r * r))
        assert cur <= prev * (1 + 1e-12)
        prev = cur


def test_hough_data_of_a_constant_sinogram():
    N = 16
    K, M = phantoms.geometry_for(N)
    c = 3.0
    hd = so.hough_data(np.full((K, M), c), N)
    sigma = slopes(N)
    for q in range(4):
        cols = np.arange(2 * N)[None, :]
        m = quarter_r(q, sigma[:, None], cols, N) + (M - 1) / 2.0
        inside = (m >= 0) & (m <= M - 1)
        want = c / np.sqrt(1.0 + sigma * sigma)[:, None] * np.ones_like(m)
        np.testing.assert_allclose(hd[q][inside], want[inside], rtol=1e-12)


def test_hough_data_of_a_disk_matches_its_projection():
    N = 64
    K, M = phantoms.geometry_for(N)
    R = 20.0
    c0 = (N - 1) / 2.0
    y, x = np.mgrid[0:N, 0:N]
    disk = (((x - c0) ** 2 + (y - c0) ** 2) <= R * R).astype(float)
    r = np.arange(M) - (M - 1) / 2.0
    sino = np.tile(2.0 * np.sqrt(np.clip(R * R - r * r, 0.0, None)), (K, 1))
    hd = so.hough_data(sino, N)
    hp = so.hough_project(disk)
    for q in range(4):
        for i in (0, N // 2, N - 1):
            m = hp[q, i] > 10
            ratio = float(np.mean(hd[q, i][m] / hp[q, i][m]))
            assert 0.97 < ratio < 1.03, (q, i, ratio)
