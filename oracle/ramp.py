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


# Other filters (the end of Sec. 3 notes that the recursive scheme applies to other FBP
# filters): the ramp |w| apodised by a window on |w| <= 1/2, w in cycles per sample.
WINDOWS = ("ram-lak", "shepp-logan", "cosine", "hamming", "hann")


def window(w, name: str) -> np.ndarray:
    """Apodisation window W(w): ram-lak 1, shepp-logan sin(pi w)/(pi w), cosine cos(pi w),
    hamming 0.54 + 0.46 cos(2 pi w), hann 0.5 + 0.5 cos(2 pi w)."""
    w = np.asarray(w, dtype=np.float64)
    if name == "ram-lak":
        return np.ones_like(w)
    if name == "shepp-logan":
        return np.sinc(w)
    if name == "cosine":
        return np.cos(np.pi * w)
    if name == "hamming":
        return 0.54 + 0.46 * np.cos(2 * np.pi * w)
    if name == "hann":
        return 0.5 + 0.5 * np.cos(2 * np.pi * w)
    raise ValueError(name)


def windowed_ramp_response(w, name: str) -> np.ndarray:
    """Ideal frequency response |w| W(w) of the apodised ramp."""
    return np.abs(np.asarray(w, dtype=np.float64)) * window(w, name)


def shepp_logan_h(n) -> np.ndarray:
    """Impulse response of |w| sin(pi w)/(pi w) on |w| <= 1/2: 2 / (pi^2 (1 - 4 n^2))."""
    nf = np.asarray(n, dtype=np.float64)
    return 2.0 / (np.pi ** 2 * (1.0 - 4.0 * nf * nf))


def cosine_h(n) -> np.ndarray:
    """Impulse response of |w| cos(pi w) on |w| <= 1/2: with a = pi (1 +- 2n),
    h(n) = sum over both a of ((-1)^n / (2a) - 1 / a^2)."""
    nf = np.asarray(n, dtype=np.float64)
    sign = np.where(np.asarray(n) % 2 == 0, 1.0, -1.0)
    out = np.zeros_like(nf)
    for a in (np.pi * (1.0 + 2.0 * nf), np.pi * (1.0 - 2.0 * nf)):
        out = out + sign / (2.0 * a) - 1.0 / (a * a)
    return out
