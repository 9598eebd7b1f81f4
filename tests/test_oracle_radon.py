"""Pins of the oracle's fast Radon transform (dyadic line sums resampled to (theta, r)).

* Each direction's class and slope reproduce the direction through the geometry's own
  quarter angles (a wrong class or slope is caught here).
* Mass: every projection of an image sums over the detector to the image's total (the
  Radon transform's zeroth moment; it fails without the sqrt(1 + sigma^2) path length).
* A centred disk and a random ellipse phantom against their closed-form sinograms (the
  phantom module's textbook line integrals): close up to the rasterisation and the dyadic
  approximation of the lines.
"""
import numpy as np

import oracle.radon as orad
import phantoms
from oracle.geometry import quarter_angle


def test_direction_classes_reproduce_theta():
    K = 97
    for k in range(K):
        theta = k * np.pi / K
        q, sigma = orad.theta_class(theta)
        assert 0.0 <= sigma <= 1.0 + 1e-12
        assert abs(float(quarter_angle(q, sigma)) - theta) < 1e-12


def test_projections_keep_the_mass():
    N = 32
    K, M = phantoms.geometry_for(N)
    f = np.random.default_rng(0).random((N, N))
    p = orad.fast_radon(f, K, M)
    np.testing.assert_allclose(p.sum(axis=1), f.sum(), rtol=1e-2)


def test_disk_matches_its_closed_form():
    N = 64
    K, M = phantoms.geometry_for(N)
    R = 20.0
    c0 = (N - 1) / 2.0
    y, x = np.mgrid[0:N, 0:N]
    disk = (((x - c0) ** 2 + (y - c0) ** 2) <= R * R).astype(float)
    p = orad.fast_radon(disk, K, M)
    r = np.arange(M) - (M - 1) / 2.0
    want = 2.0 * np.sqrt(np.clip(R * R - r * r, 0.0, None))
    m = want > 5
    ratio = p[:, m].mean(axis=1) / want[m].mean()
    assert np.all(np.abs(ratio - 1.0) < 0.03), ratio
    assert np.median(np.abs(p[:, m] - want[m]) / want[m]) < 0.02


def test_ellipse_phantom_matches_its_closed_form():
    N = 64
    K, M = phantoms.geometry_for(N)
    ell = phantoms.random_ellipses(7)
    p = orad.fast_radon(phantoms.ellipse_image(ell, N), K, M)
    want = phantoms.ellipse_sinogram(ell, N, K, M)
    assert np.linalg.norm(p - want) / np.linalg.norm(want) < 0.06
