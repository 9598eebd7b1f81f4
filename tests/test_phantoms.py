"""Pins of the synthetic input generator (textbook ellipse Radon transform)."""
import math

import numpy as np
import pytest

import phantoms


def _line_integral(ellipses, theta, R, n=400_001):
    # numerical integral of the density along {X cos + Y sin = R}, t in [-2, 2]
    t = np.linspace(-2.0, 2.0, n)
    X = R * np.cos(theta) - t * np.sin(theta)
    Y = R * np.sin(theta) + t * np.cos(theta)
    dens = np.zeros_like(t)
    for e in ellipses:
        dx, dy = X - e.x0, Y - e.y0
        u = (dx * math.cos(e.alpha) + dy * math.sin(e.alpha)) / e.a
        v = (-dx * math.sin(e.alpha) + dy * math.cos(e.alpha)) / e.b
        dens += np.where(u * u + v * v <= 1, e.rho, 0.0)
    return np.trapezoid(dens, t)


def test_closed_form_matches_numerical_line_integrals():
    ell = phantoms.random_ellipses(123)
    rng = np.random.default_rng(0)
    th = rng.uniform(0, np.pi, 12)
    R = rng.uniform(-0.9, 0.9, 12)
    closed = np.array([phantoms._norm_sinogram(ell, np.array([a]), np.array([r]))[0, 0]
                       for a, r in zip(th, R)])
    numeric = np.array([_line_integral(ell, a, r) for a, r in zip(th, R)])
    np.testing.assert_allclose(closed, numeric, atol=2e-4)


def test_mass_is_the_same_in_every_projection():
    N = 128
    K, M = phantoms.geometry_for(N)
    ell = phantoms.random_ellipses(77)
    s = phantoms.ellipse_sinogram(ell, N, K, M)
    mass = sum(e.rho * math.pi * e.a * e.b for e in ell) * (N / 2) ** 2   # pixel units
    np.testing.assert_allclose(s.sum(axis=1), mass, rtol=2e-3)


def test_recipe_ranges_and_seeding():
    a = phantoms.random_ellipses(2020)
    b = phantoms.random_ellipses(2020)
    assert a == b and len(a) == 10
    for e in a:
        assert math.hypot(e.x0, e.y0) <= 0.8
        assert 0.05 <= e.a <= 0.5 and 0.05 <= e.b <= 0.5
        assert 0 <= e.alpha < math.pi and -0.5 <= e.rho <= 1.0
    assert phantoms.geometry_for(2048) == (3072, 2897)
    assert phantoms.geometry_for(256) == (384, 363)


def test_poisson_noise_is_unbiased_in_counts():
    p = np.full((200, 200), 0.7)
    noisy = phantoms.poisson_log_noise(p, 1e5, 4)
    assert abs(np.exp(-noisy).mean() - np.exp(-0.7)) < 1e-3 * np.exp(-0.7)
