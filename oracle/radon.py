"""Fast (approximate) Radon transform: the dyadic line sums of the fast Hough transform
(Eq. 17: the projection in (s, t) coordinates, one pixel per row along each line) resampled
to an ordinary (theta, r) sinogram.

TEST INFRASTRUCTURE ONLY (see the package docstring).

For sinogram row k, theta_k = k pi / K lies in one line class (geometry module):
    [0, pi/4]      v-  sigma = tan(theta)
    (pi/4, pi/2]   h-  sigma = tan(pi/2 - theta)
    (pi/2, 3pi/4]  h+  sigma = tan(theta - pi/2)
    (3pi/4, pi)    v+  sigma = tan(pi - theta)
(each shared end direction taken by the first class listed).  The fractional linogram row
is i* = sigma (N - 1), between rows i0 = min(floor(i*), N - 2) and i0 + 1, weight
t = i* - i0.  In each of the two rows the detector offset r_m = m - (M-1)/2 falls at the
stored column c where the row's line has offset r (quarter_r is affine in c); the row is
read there by linear interpolation in c (zero outside [0, 2N)).  The two values are mixed
with weights (1 - t, t), and multiplied by the path length per row sqrt(1 + sigma^2), since
a dyadic line sum counts one pixel per row while the Radon transform integrates along the
line.
"""
from __future__ import annotations

import numpy as np

from .geometry import quarter_r
from .sirt import hough_project


def theta_class(theta: float):
    """(quarter q, slope sigma) of the line class holding direction theta in [0, pi)."""
    if theta <= np.pi / 4:
        return 0, np.tan(theta)
    if theta <= np.pi / 2:
        return 2, np.tan(np.pi / 2 - theta)
    if theta <= 3 * np.pi / 4:
        return 3, np.tan(theta - np.pi / 2)
    return 1, np.tan(np.pi - theta)


def _row_at_offsets(Hrow, q: int, sigma: float, r, N: int) -> np.ndarray:
    """Linear interpolation of one linogram row at the columns of detector offsets r."""
    r0 = quarter_r(q, sigma, 0.0, N)
    dr = quarter_r(q, sigma, 1.0, N) - r0            # r is affine in the column
    c = (np.asarray(r, np.float64) - r0) / dr
    W = Hrow.shape[0]
    c0 = np.floor(c)
    f = c - c0
    c0 = c0.astype(np.int64)

    def at(j):
        ok = (j >= 0) & (j < W)
        return np.where(ok, Hrow[np.clip(j, 0, W - 1)], 0.0)

    return (1.0 - f) * at(c0) + f * at(c0 + 1)


def radon_from_hough(H, N: int, K: int, M: int) -> np.ndarray:
    """Sinogram [K][M] (float64) from dyadic line sums H [4][N][2N]."""
    H = np.asarray(H, np.float64)
    r = np.arange(M, dtype=np.float64) - (M - 1) / 2.0
    out = np.zeros((K, M))
    for k in range(K):
        q, sigma = theta_class(k * np.pi / K)
        istar = sigma * (N - 1)
        i0 = min(int(np.floor(istar)), N - 2)
        t = istar - i0
        v0 = _row_at_offsets(H[q, i0], q, i0 / (N - 1), r, N)
        v1 = _row_at_offsets(H[q, i0 + 1], q, (i0 + 1) / (N - 1), r, N)
        out[k] = ((1.0 - t) * v0 + t * v1) * np.sqrt(1.0 + sigma * sigma)
    return out


def fast_radon(f, K: int, M: int) -> np.ndarray:
    """The fast Radon transform of an image f [N][N] (float64)."""
    f = np.asarray(f, np.float64)
    return radon_from_hough(hough_project(f), f.shape[0], K, M)
