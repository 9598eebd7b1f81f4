"""Pins of the ramp kernel (Sec. 3, Eq. 6, 7, 10) against quadrature and the DTFT."""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle import anticausal_part, causal_part, ramp_h, ramp_h_sinc


def test_eq7_equals_band_limited_integral():
    # Eq. 6 as an integral: h(n) = 2 * int_0^{1/2} w cos(2 pi w n) dw, by quadrature.
    for n in range(-15, 16):
        val, _ = quad(lambda w: 2.0 * w * np.cos(2 * np.pi * w * n), 0.0, 0.5, epsabs=1e-14)
        assert ramp_h(n) == pytest.approx(val, abs=1e-13)


def test_eq7_equals_sinc_form_of_eq6():
    n = np.arange(-60, 61)
    np.testing.assert_allclose(ramp_h(n), ramp_h_sinc(n), atol=1e-15)


def test_dtft_is_ramp():
    # sum_n h(n) e^{-2 pi i w n} = |w| on |w| <= 1/2 (truncation at |n| <= T costs <= 2/(pi^2 T)).
    T = 400_001
    n = np.arange(1, T)
    h = ramp_h(n)
    for w in (0.0, 0.03, 0.1, 0.25, 0.37, 0.5):
        H = ramp_h(0) + 2.0 * np.sum(h * np.cos(2 * np.pi * w * n))
        assert H == pytest.approx(abs(w), abs=2.0 / (np.pi ** 2 * T) + 1e-12)


def test_causal_anticausal_split_eq10():
    n = np.arange(-30, 31)
    np.testing.assert_array_equal(causal_part(n) + anticausal_part(n), ramp_h(n))
    np.testing.assert_array_equal(causal_part(n), anticausal_part(-n))
    assert causal_part(0) == 0.125 and causal_part(-3) == 0.0
