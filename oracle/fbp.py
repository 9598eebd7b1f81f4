"""The whole fast method and the direct FBP (paper Sec. 2-5).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Fast method (Conclusion; Eq. 12 -> 14 -> 21 -> 22): recursive ramp filtering of every
projection, resampling into the four linogram quarters, back projection of each quarter
along dyadic patterns, sum of the four quarter images.

Direct FBP (Eq. 3-5 with Eq. 8): the exact FIR ramp filter followed by pixel-driven
back projection with linear interpolation along the detector,
    f(x, y) = (pi / K) * sum_k p~_k((x - c0) cos(theta_k) + (y - c0) sin(theta_k)).
Reading fixed here: Eq. 5 integrates over [0, 2 pi) but a parallel-beam sinogram covers
[0, pi); the integral is taken over [0, pi) with K uniform angles, i.e. weight pi / K.
"""
from __future__ import annotations

import numpy as np

from .dyadic import combine_quarters, dyadic_pattern, fht_stages, pattern_backproject, _log2
from .iir import fir_ramp, iir_filter
from .linogram import linogram, linogram_at


def _check(sino, N):
    sino = np.asarray(sino, dtype=np.float64)
    if sino.ndim != 2:
        raise ValueError("one sinogram [K][M] at a time")
    _log2(N)
    return sino


def fast_fbp(sino, N: int, b, a, backproject: str = "pattern") -> np.ndarray:
    """Fast reconstruction of one slice, float64 unless ``backproject == 'fht32'``.

    backproject: 'pattern' sums each dyadic pattern directly (no recursion); 'fht64' and
    'fht32' use the stage recursion in float64 / float32.
    """
    sino = _check(sino, N)
    return fast_backproject(iir_filter(sino, b, a), N, backproject)


def fast_backproject(pt, N: int, backproject: str = "pattern") -> np.ndarray:
    """Resampling, quarter back projection and quarter sum of an already filtered sinogram."""
    pt = _check(pt, N)
    L = linogram(pt, N)
    if backproject == "pattern":
        F = np.stack([pattern_backproject(L[q]) for q in range(4)])
    elif backproject == "fht64":
        F = np.stack([fht_stages(L[q], np.float64) for q in range(4)])
    elif backproject == "fht32":
        return fht_backproject(L.astype(np.float32))
    else:
        raise ValueError(backproject)
    return combine_quarters(F)


def fht_backproject(lin) -> np.ndarray:
    """float32 back projection of a linogram [4][N][W] (W >= 2N-1): the stage recursion
    per quarter, then the Eq. 22 sum in its fixed order, all in float32."""
    lin = np.asarray(lin, dtype=np.float32)
    F = np.stack([fht_stages(lin[q], np.float32) for q in range(4)])
    return combine_quarters(F)


def fast_fbp_pixels(sino, N: int, b, a, ys, xs, pt=None) -> np.ndarray:
    """The 'pattern' fast reconstruction at the pixels (ys[j], xs[j]) only (float64).

    The linogram samples each pattern visits are evaluated on demand, so this runs at any
    N.  ``pt`` may pass a precomputed IIR-filtered sinogram.
    """
    sino = _check(sino, N)
    n = _log2(N)
    if pt is None:
        pt = iir_filter(sino, b, a)
    ys = np.asarray(ys, dtype=np.int64)
    xs = np.asarray(xs, dtype=np.int64)
    rows = np.arange(N)
    out = np.empty(ys.size)
    for j, (y, x) in enumerate(zip(ys, xs)):
        dy, dx = dyadic_pattern(n, int(y)), dyadic_pattern(n, int(x))
        fv_minus = linogram_at(pt, 0, rows, x + dy, N).sum()
        fv_plus = linogram_at(pt, 1, rows, (N - 1 - x) + dy, N).sum()
        fh_minus = linogram_at(pt, 2, rows, y + dx, N).sum()
        fh_plus = linogram_at(pt, 3, rows, (N - 1 - y) + dx, N).sum()
        out[j] = (fv_minus + fv_plus) + (fh_minus + fh_plus)
    return out


def _backproject_direct(pt, N, ys, xs):
    K, M = pt.shape
    c0 = (N - 1) / 2.0
    X = np.asarray(xs, dtype=np.float64) - c0
    Y = np.asarray(ys, dtype=np.float64) - c0
    acc = np.zeros(np.broadcast(X, Y).shape)
    for k in range(K):
        th = k * np.pi / K
        m = X * np.cos(th) + Y * np.sin(th) + (M - 1) / 2.0
        j0 = np.floor(m)
        f = m - j0
        j0 = j0.astype(np.int64)
        row = pt[k]
        v0 = np.where((j0 >= 0) & (j0 < M), row[np.clip(j0, 0, M - 1)], 0.0)
        v1 = np.where((j0 + 1 >= 0) & (j0 + 1 < M), row[np.clip(j0 + 1, 0, M - 1)], 0.0)
        acc += (1.0 - f) * v0 + f * v1
    return acc * (np.pi / K)


def direct_fbp(sino, N: int) -> np.ndarray:
    """Direct Theta(N^3) reconstruction of one slice (float64), image [y][x]."""
    sino = _check(sino, N)
    pt = fir_ramp(sino)
    y, x = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    return _backproject_direct(pt, N, y, x)


def direct_fbp_pixels(sino, N: int, ys, xs, pt=None) -> np.ndarray:
    """Direct reconstruction at the pixels (ys[j], xs[j]) only."""
    sino = _check(sino, N)
    if pt is None:
        pt = fir_ramp(sino)
    return _backproject_direct(pt, N, np.asarray(ys), np.asarray(xs))
