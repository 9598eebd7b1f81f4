"""Resampling of the filtered sinogram into the four linogram quarters
(paper Sec. 4.2, Eq. 14-15).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings fixed here:
* "Linear interpolation" is bilinear in (angle index, detector index): the angle index of
  theta is theta*K/pi, the detector index of r is r + (M-1)/2.
* Detector samples outside [0, M) are zero.
* Between the last angle theta_{K-1} and pi the second sample is taken at angle 0 with the
  detector mirrored, because p(theta + pi, r) = p(theta, -r).
* L_q[i][c] = w_i * p~(theta_q(sigma_i), r_q(sigma_i, c)), with w_i the row weight of the
  geometry module.  The array is stored with width 2N.
"""
from __future__ import annotations

import numpy as np

from .geometry import quarter_angle, quarter_r, row_weights


def _row_lerp(pt, rows, m):
    """Linear interpolation along the detector of rows ``rows`` at index m, zero outside."""
    M = pt.shape[-1]
    j0 = np.floor(m)
    f = m - j0
    j0 = j0.astype(np.int64)
    j1 = j0 + 1
    v0 = np.where((j0 >= 0) & (j0 < M), pt[rows, np.clip(j0, 0, M - 1)], 0.0)
    v1 = np.where((j1 >= 0) & (j1 < M), pt[rows, np.clip(j1, 0, M - 1)], 0.0)
    return (1.0 - f) * v0 + f * v1


def sample_filtered(pt, theta, r) -> np.ndarray:
    """Bilinear value of the sinogram ``pt`` [K][M] at angle theta in [0, pi] and offset r."""
    pt = np.asarray(pt, dtype=np.float64)
    K, M = pt.shape
    theta, r = np.broadcast_arrays(np.asarray(theta, np.float64), np.asarray(r, np.float64))
    tk = theta * K / np.pi
    k0 = np.minimum(np.floor(tk), K - 1)
    ft = tk - k0
    k0 = k0.astype(np.int64)
    m = r + (M - 1) / 2.0
    va = _row_lerp(pt, k0, m)
    k1 = k0 + 1
    wrap = k1 >= K
    vb = _row_lerp(pt, np.where(wrap, 0, k1), np.where(wrap, (M - 1) - m, m))
    return (1.0 - ft) * va + ft * vb


def linogram_at(pt, q: int, i, c, N: int) -> np.ndarray:
    """L_q[i][c] for integer arrays i (slope rows) and c (stored columns)."""
    i = np.asarray(i)
    sigma = i / (N - 1)
    theta = quarter_angle(q, sigma)
    r = quarter_r(q, sigma, c, N)
    return row_weights(N)[i] * sample_filtered(pt, theta, r)


def linogram(pt, N: int) -> np.ndarray:
    """The four quarters [4][N][2N] (float64), quarter order v-, v+, h-, h+."""
    i = np.arange(N)[:, None]
    c = np.arange(2 * N)[None, :]
    return np.stack([linogram_at(pt, q, i, c, N) for q in range(4)])
