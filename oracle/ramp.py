"""Band-limited discrete ramp kernel (paper Sec. 3, Eq. 6, 7 and 10).

TEST INFRASTRUCTURE ONLY (see the package docstring).

With the detector spacing set to 1, the band limit is |omega| < 1/2 and the ideal ramp
|omega| has the impulse response h(n) = 2 * int_0^{1/2} omega cos(2 pi omega n) d omega.
"""
from __future__ import annotations

import numpy as np


def ramp_h(n) -> np.ndarray:
    """Eq. 7: h(0) = 1/4, h(n) = 0 for even n != 0, h(n) = -1/(pi n)^2 for odd n."""
    n = np.asarray(n)
    nf = n.astype(np.float64)
    out = np.zeros(n.shape, dtype=np.float64)
    out[n == 0] = 0.25
    odd = (n % 2) != 0
    out[odd] = -1.0 / (np.pi * nf[odd]) ** 2
    return out


def ramp_h_sinc(n) -> np.ndarray:
    """Eq. 6: h(n) = sinc(pi n)/2 - sinc^2(pi n/2)/4 with sinc(r) = sin(r)/r.

    numpy's ``sinc(x)`` is sin(pi x)/(pi x), so the paper's sinc(pi n) is ``np.sinc(n)``.
    """
    nf = np.asarray(n, dtype=np.float64)
    return np.sinc(nf) / 2.0 - np.sinc(nf / 2.0) ** 2 / 4.0


def causal_part(n) -> np.ndarray:
    """Eq. 10, h+: h(0)/2 at n = 0, h(n) for n > 0, zero for n < 0."""
    n = np.asarray(n)
    out = np.where(n > 0, ramp_h(n), 0.0)
    return np.where(n == 0, ramp_h(0) / 2.0, out)


def anticausal_part(n) -> np.ndarray:
    """Eq. 10, h-: h(0)/2 at n = 0, h(n) for n < 0, zero for n > 0."""
    n = np.asarray(n)
    out = np.where(n < 0, ramp_h(n), 0.0)
    return np.where(n == 0, ramp_h(0) / 2.0, out)
