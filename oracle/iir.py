"""Recursive (IIR) ramp filtering and the exact FIR ramp (paper Sec. 3, Eq. 8, 9, 12, 13).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings fixed here:
* Eq. 13 prints the full output p~ in the feedback sum; a recursive filter feeds back its
  own past output (Eq. 9), so the causal branch feeds back p~+ and the anticausal branch
  p~-.  The coefficients are shared: a+ = a-, b+ = b- (text after Eq. 13).
* The paper is silent on the boundary.  Each projection row is filtered with zero state:
  the signal and both filter outputs are zero outside [0, M).
* Eq. 8's summation bounds are garbled; the FIR is read as sum over k in [-L0, L0] of
  h(k) p(n - k) with p = 0 outside the row.  With L0 = M - 1 it is the exact linear
  convolution of the row with h.

Arrays hold one projection per row: the filter runs along the last axis.
"""
from __future__ import annotations

import numpy as np

from .ramp import ramp_h


def iir_causal(p, b, a) -> np.ndarray:
    """Eq. 13 (upper signs): y(n) = sum_{k<Mb} b_k p(n-k) - sum_{k=1..Q} a_k y(n-k)."""
    p = np.asarray(p, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    M = p.shape[-1]
    y = np.zeros_like(p)
    for n in range(M):
        acc = np.zeros(p.shape[:-1])
        for k in range(b.size):
            if n - k >= 0:
                acc = acc + b[k] * p[..., n - k]
        for k in range(1, a.size + 1):
            if n - k >= 0:
                acc = acc - a[k - 1] * y[..., n - k]
        y[..., n] = acc
    return y


def iir_anticausal(p, b, a) -> np.ndarray:
    """Eq. 13 (lower signs): y(n) = sum_{k<Mb} b_k p(n+k) - sum_{k=1..Q} a_k y(n+k)."""
    p = np.asarray(p, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    M = p.shape[-1]
    y = np.zeros_like(p)
    for n in range(M - 1, -1, -1):
        acc = np.zeros(p.shape[:-1])
        for k in range(b.size):
            if n + k < M:
                acc = acc + b[k] * p[..., n + k]
        for k in range(1, a.size + 1):
            if n + k < M:
                acc = acc - a[k - 1] * y[..., n + k]
        y[..., n] = acc
    return y


def iir_filter(p, b, a) -> np.ndarray:
    """Eq. 12: p~ = p~+ + p~-, the ramp-filtered projection."""
    return iir_causal(p, b, a) + iir_anticausal(p, b, a)


def iir_impulse_response(b, a, length: int) -> np.ndarray:
    """Causal impulse response g(0..length-1) of the Eq. 9 difference equation."""
    delta = np.zeros(length)
    delta[0] = 1.0
    return iir_causal(delta, b, a)


def fir_ramp(p) -> np.ndarray:
    """Eq. 8 with L0 = M - 1: exact convolution of each row with the Eq. 7 kernel.

    The linear convolution is evaluated with an FFT (a library primitive); the kernel
    taps are h(k) for k in [-(M-1), M-1].
    """
    p = np.asarray(p, dtype=np.float64)
    M = p.shape[-1]
    k = np.arange(-(M - 1), M)
    h = ramp_h(k)
    nfft = 1
    while nfft < 3 * M - 2:
        nfft *= 2
    full = np.fft.irfft(np.fft.rfft(p, nfft, axis=-1) * np.fft.rfft(h, nfft), nfft, axis=-1)
    # full[j] = sum_k h[k + M - 1] p[j - (k + M - 1)]; output n corresponds to j = n + M - 1.
    return full[..., M - 1:2 * M - 1]
