"""Pins of the recursive filters (Eq. 9, 12, 13) and the exact FIR (Eq. 8)."""
import numpy as np
import pytest
from scipy.signal import lfilter, residuez

from oracle import (fir_ramp, iir_anticausal, iir_causal, iir_filter, iir_impulse_response,
                    ramp_h)

RNG = np.random.default_rng(11)
B3 = np.array([0.12, -0.23, 0.11])


def test_no_feedback_is_textbook_convolution():
    p = RNG.normal(size=(3, 40))
    b = RNG.normal(size=4)
    got = iir_causal(p, b, [])
    want = np.stack([np.convolve(r, b)[:40] for r in p])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


def test_single_pole_closed_form():
    rho, b0, b1 = 0.8, 0.7, -0.2
    g = iir_impulse_response([b0, b1], [-rho], 30)
    n = np.arange(30)
    want = b0 * rho ** n + np.where(n >= 1, b1 * rho ** (n - 1.0), 0.0)
    np.testing.assert_allclose(g, want, rtol=1e-13, atol=1e-15)


def test_third_order_partial_fractions():
    # Impulse response from the residues and poles of B(z)/A(z) (scipy.signal.residuez).
    a_full = np.poly([0.9, 0.5, -0.3])
    r, p, k = residuez(B3, a_full)
    n = np.arange(60)
    want = np.real(sum(ri * pi ** n for ri, pi in zip(r, p)))
    for j, kj in enumerate(np.atleast_1d(k)):
        want[j] += np.real(kj)
    got = iir_impulse_response(B3, a_full[1:], 60)
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-13)


def test_matches_library_difference_equation():
    a_full = np.poly([0.95, 0.4, -0.6])
    p = RNG.normal(size=(4, 200))
    np.testing.assert_allclose(iir_causal(p, B3, a_full[1:]), lfilter(B3, a_full, p, axis=-1),
                               rtol=1e-11, atol=1e-12)


def test_anticausal_is_time_reversed_causal():
    a = np.poly([0.9, 0.5, -0.3])[1:]
    p = RNG.normal(size=(2, 77))
    np.testing.assert_allclose(iir_anticausal(p, B3, a), iir_causal(p[:, ::-1], B3, a)[:, ::-1],
                               rtol=0, atol=1e-13)


def test_fused_filter_is_symmetric_fir_of_impulse_response():
    # Eq. 12: p~ = p * g(n) + p * g(-n), i.e. a symmetric FIR with tap 2 g(0) at the centre.
    a = np.poly([0.9, 0.5, -0.3])[1:]
    g = iir_impulse_response(B3, a, 10_000)
    M = 120
    p = RNG.normal(size=M)
    kern = np.concatenate([g[1:M][::-1], [2 * g[0]], g[1:M]])      # taps -(M-1)..(M-1)
    want = np.convolve(p, kern)[M - 1:2 * M - 1]
    np.testing.assert_allclose(iir_filter(p[None], B3, a)[0], want, rtol=0, atol=1e-12)


def test_fir_ramp_brute_force():
    M = 23
    p = RNG.normal(size=(2, M))
    want = np.zeros_like(p)
    for n in range(M):
        for k in range(-(M - 1), M):
            if 0 <= n - k < M:
                want[:, n] += ramp_h(k) * p[:, n - k]
    np.testing.assert_allclose(fir_ramp(p), want, rtol=0, atol=1e-13)


def test_fir_ramp_of_delta_is_kernel():
    M = 31
    p = np.zeros((1, M))
    p[0, 10] = 1.0
    np.testing.assert_allclose(fir_ramp(p)[0], ramp_h(np.arange(M) - 10), atol=1e-15)


@pytest.mark.parametrize("N", [256, 2048])
def test_committed_table_filters_are_stable_and_dc_free(coeff_table, N):
    for e in coeff_table["entries"]:
        if e["N"] != N:
            continue
        poles = np.roots(np.concatenate([[1.0], e["a"]]))
        assert np.abs(poles).max() < 0.99999
        assert abs(sum(e["b"])) < 1e-12
