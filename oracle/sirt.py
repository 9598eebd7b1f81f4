"""Algebraic reconstruction on the fast Hough operators: the FHT-based iterative method that
the paper points to beside its fast FBP (Sec. 4.4: a fast SART built on the fast Hough
transform, after Prun et al.), in its simultaneous form (SIRT).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Operators (float64, brute force over the dyadic patterns of Sec. 4.3):
  A f   the dyadic line sums of an image, [4][N][2N]: line (q, i, c) of quarter q, slope
        i/(N-1), stored intercept c (the '+' quarters flipped as in the back projection).
        It is the transpose of the quarter back projection + Eq. 22 sum (adjoint module).
  A^T L the back projection of a linogram: the brute-force pattern sums per quarter, then
        the Eq. 22 sum.
SIRT: f_{k+1} = f_k + lam C^-1 A^T (R^-1 (b - A f_k)) with R = A 1 (pixels on each line)
and C = A^T 1 (lines through each pixel); entries where R or C is zero contribute nothing.
For 0 < lam < 2 the iteration decreases the R^-1-weighted residual and, for consistent
data of a full-rank system, converges to the image that produced it.

Hough-space data of a sinogram: a dyadic line visits one pixel per row of its quarter, so
its pixel sum approximates the line integral divided by the path length per row,
sqrt(1 + sigma^2).  The data are the sinogram sampled bilinearly at the linogram points
(Eq. 14-15) divided by that length: hough_data(p) = linogram(p) / (w_i sqrt(1 + sigma_i^2)),
w_i the linogram row weights (which the FBP integral needs and SIRT does not).
"""
from __future__ import annotations

import numpy as np

from .adjoint import fht_backproject_adjoint
from .dyadic import combine_quarters, pattern_backproject
from .geometry import row_weights, slopes
from .linogram import linogram


def hough_project(f) -> np.ndarray:
    """A f: image [N][N] -> dyadic line sums [4][N][2N] (float64)."""
    return fht_backproject_adjoint(np.asarray(f, np.float64), brute=True)


def back_project(L) -> np.ndarray:
    """A^T L: linogram [4][N][W] -> image [N][N] (float64)."""
    L = np.asarray(L, np.float64)
    return combine_quarters(np.stack([pattern_backproject(L[q]) for q in range(4)]))


def sirt_weights(N: int):
    """(R^-1, C^-1): reciprocals of A 1 and A^T 1, zero where those vanish."""
    R = hough_project(np.ones((N, N)))
    C = back_project(np.ones((4, N, 2 * N)))
    rinv = np.divide(1.0, R, out=np.zeros_like(R), where=R > 0)
    cinv = np.divide(1.0, C, out=np.zeros_like(C), where=C > 0)
    return rinv, cinv


def sirt(b, N: int, iters: int, lam: float, f0=None) -> np.ndarray:
    """`iters` SIRT steps on data b [4][N][2N] from f0 (zero by default)."""
    rinv, cinv = sirt_weights(N)
    f = np.zeros((N, N)) if f0 is None else np.array(f0, np.float64)
    b = np.asarray(b, np.float64)
    for _ in range(iters):
        f = f + lam * cinv * back_project(rinv * (b - hough_project(f)))
    return f


def hough_data(sino, N: int) -> np.ndarray:
    """Hough-space data [4][N][2N] of a sinogram [K][M] (float64)."""
    sigma = slopes(N)
    scale = 1.0 / (row_weights(N) * np.sqrt(1.0 + sigma * sigma))
    return linogram(np.asarray(sino, np.float64), N) * scale[None, :, None]
