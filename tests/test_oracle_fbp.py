"""Pins of the whole fast method and of the direct FBP (Sec. 2, 5; Eq. 5, 16, 22)."""
import numpy as np
import pytest

import phantoms
from oracle import (direct_fbp, fast_backproject, fast_fbp, fast_fbp_pixels, fir_ramp,
                    iir_filter)

B = np.array([0.12, -0.23, 0.11])
A = np.poly([0.9, 0.5, -0.3])[1:]


def _disk(N, rho=1.0, R=0.6, x0=0.0, y0=0.0):
    K, M = phantoms.geometry_for(N)
    return phantoms.ellipse_sinogram([phantoms.Ellipse(x0, y0, R, R, 0.0, rho)], N, K, M)


@pytest.mark.parametrize("N", [64, 128])
def test_uniform_disk_reconstructs_to_its_density(N):
    # A centred disk of density 1.7: the interior of both reconstructions (with the exact
    # ramp) is 1.7 to within the discretisation error of the sampled transform.
    s = _disk(N, rho=1.7)
    c = slice(N // 2 - N // 16, N // 2 + N // 16)
    fd = direct_fbp(s, N)
    ff = fast_backproject(fir_ramp(s), N)
    assert fd[c, c].mean() == pytest.approx(1.7, rel=3e-3)
    assert ff[c, c].mean() == pytest.approx(1.7, rel=3e-3)


def test_fast_back_projection_tracks_direct_on_asymmetric_phantom():
    # Off-centre, rotated ellipses: any quarter mapped to the wrong pixels (a missing flip
    # or transpose) makes the fast image far from the direct one.
    N = 64
    K, M = phantoms.geometry_for(N)
    ell = phantoms.random_ellipses(4)
    s = phantoms.ellipse_sinogram(ell, N, K, M)
    pt = fir_ramp(s)
    fd = direct_fbp(s, N)
    ff = fast_backproject(pt, N)
    rng = fd.max() - fd.min()
    assert np.sqrt(np.mean((ff - fd) ** 2)) < 0.03 * rng
    # a deliberately mis-mapped variant is far off, so the bound above is discriminating
    assert np.sqrt(np.mean((ff.T - fd) ** 2)) > 0.1 * rng


def test_transposed_object_gives_transposed_image_eq16():
    # Transposing the object maps the line (theta, r) to (pi/2 - theta, r); with K even
    # that permutes the sinogram rows (with r -> -r past pi).  The h quarters are the v
    # quarters of the transposed image (Eq. 16), so the result must be the transpose.
    N = 32
    K, M = phantoms.geometry_for(N)
    rng = np.random.default_rng(3)
    s = rng.normal(size=(K, M))
    sT = np.empty_like(s)
    for kp in range(K):
        if kp <= K // 2:
            sT[kp] = s[K // 2 - kp]
        else:
            sT[kp] = s[3 * K // 2 - kp][::-1]
    f = fast_fbp(s, N, B, A)
    fT = fast_fbp(sT, N, B, A)
    np.testing.assert_allclose(fT, f.T, rtol=0, atol=1e-12)


def test_linearity():
    N = 16
    K, M = phantoms.geometry_for(N)
    rng = np.random.default_rng(9)
    s1, s2 = rng.normal(size=(2, K, M))
    lhs = fast_fbp(2.5 * s1 - 0.75 * s2, N, B, A)
    rhs = 2.5 * fast_fbp(s1, N, B, A) - 0.75 * fast_fbp(s2, N, B, A)
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-12)


def test_pixel_subset_and_recursions_agree_with_brute_force():
    N = 32
    K, M = phantoms.geometry_for(N)
    s = phantoms.ellipse_sinogram(phantoms.random_ellipses(7), N, K, M)
    f = fast_fbp(s, N, B, A)
    np.testing.assert_allclose(fast_fbp(s, N, B, A, "fht64"), f, rtol=0, atol=1e-12)
    f32 = fast_fbp(s, N, B, A, "fht32")
    assert np.abs(f32 - f).max() < 1e-6 * (f.max() - f.min())
    ys = np.array([0, 5, 31, 17, 31])
    xs = np.array([0, 30, 31, 2, 0])
    np.testing.assert_allclose(fast_fbp_pixels(s, N, B, A, ys, xs), f[ys, xs], rtol=0, atol=1e-12)


def test_direct_fbp_of_single_projection_is_a_smeared_line():
    # One nonzero projection at theta_k: the back projection is constant along lines of
    # that angle; at theta = 0 every image column x carries pt[0](x - c0).
    N = 16
    K, M = phantoms.geometry_for(N)
    s = np.zeros((K, M))
    s[0] = np.random.default_rng(1).normal(size=M)
    f = direct_fbp(s, N)
    pt = fir_ramp(s)[0]
    c0 = (N - 1) / 2
    for x in range(N):
        m = (x - c0) + (M - 1) / 2
        j = int(np.floor(m))
        val = (1 - (m - j)) * pt[j] + (m - j) * pt[j + 1]
        np.testing.assert_allclose(f[:, x], np.full(N, val * np.pi / K), atol=1e-13)
