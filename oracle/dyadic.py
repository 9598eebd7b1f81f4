"""Dyadic patterns and the fast Hough transform back projection (paper Sec. 4.3-4.5,
Eq. 16-22).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings fixed here (the paper cites the dyadic-pattern algorithm but does not restate it):
* N is a power of two, N = 2^n.
* The dyadic pattern of slope tau over 2^n rows, d_tau(i) for i in [0, 2^n), is defined
  recursively: the pattern over one row is (0); the pattern of slope tau over 2^n rows is
  the pattern of slope floor(tau/2) over the first 2^(n-1) rows, followed by the same
  pattern shifted right by ceil(tau/2) over the last 2^(n-1) rows.  So d_tau(0) = 0,
  d_tau(2^n - 1) = tau, and each step is 0 or 1.
* Back projection of one linogram quarter (Eq. 19-21, Brady's approach): the quarter image
  is F[tau][u] = sum_i L[i][u + d_tau(i)] for tau, u in [0, N); the pixel mapping of each
  quarter is in ``combine_quarters``.
* The fast transform evaluates these sums by log2(N) stages of pair additions.  Stage k
  merges strips 2b and 2b+1 (height 2^(k-1)) into strip b:
      H_k[b][tau][u] = H_{k-1}[2b][floor(tau/2)][u] + H_{k-1}[2b+1][floor(tau/2)][u + ceil(tau/2)]
  with H_0[i][0][u] = L[i][u] and columns at or beyond the stored width read as zero.
* Eq. 22 sums the four quarter images; the order of the sum is fixed here as
  (F_v- + F_v+) + (F_h- + F_h+) so that float32 results are reproducible bit for bit.
"""
from __future__ import annotations

import numpy as np


def dyadic_pattern(n: int, tau: int) -> np.ndarray:
    """d_tau(i), i in [0, 2^n), by the recursive definition in the module docstring."""
    if n == 0:
        return np.zeros(1, dtype=np.int64)
    half = dyadic_pattern(n - 1, tau // 2)
    return np.concatenate([half, half + (tau + 1) // 2])


def _log2(N: int) -> int:
    n = N.bit_length() - 1
    if N < 1 or (1 << n) != N:
        raise ValueError("N must be a power of two")
    return n


def pattern_backproject(Lq, taus=None) -> np.ndarray:
    """Brute-force sums F[tau][u] = sum_i L[i][u + d_tau(i)] (float64), i ascending.

    ``taus`` restricts the output to those slopes (rows of the result, in that order)."""
    Lq = np.asarray(Lq, dtype=np.float64)
    N, W = Lq.shape
    n = _log2(N)
    u = np.arange(N)
    rows = np.arange(N)
    taus = range(N) if taus is None else list(taus)
    F = np.empty((len(taus), N))
    for j, tau in enumerate(taus):
        cols = u[:, None] + dyadic_pattern(n, tau)[None, :]       # [u][i]
        vals = np.where(cols < W, Lq[rows[None, :], np.minimum(cols, W - 1)], 0.0)
        F[j] = vals.sum(axis=1)
    return F


def fht_stages(Lq, dtype=np.float32) -> np.ndarray:
    """The stage recursion of the module docstring, evaluated in ``dtype``.

    Returns H[tau][u] for tau, u in [0, N).  In float32 every stage result is rounded to
    float32 (numpy adds are IEEE round-to-nearest-even), which fixes the value of every
    partial sum, so an implementation that performs the same additions reproduces the
    output bit for bit whatever order it performs them in.
    """
    Lq = np.asarray(Lq, dtype=dtype)
    N, W = Lq.shape
    n = _log2(N)
    H = Lq.reshape(N, 1, W)                      # [strip b][tau][u], strips of one row
    for k in range(1, n + 1):
        h = 1 << k
        new = np.empty((N >> k, h, W), dtype=dtype)
        for tau in range(h):
            top = H[0::2, tau // 2, :]
            bot = H[1::2, tau // 2, :]
            s = (tau + 1) // 2
            shifted = np.zeros_like(bot)
            shifted[:, :W - s] = bot[:, s:]
            new[:, tau, :] = top + shifted
        H = new
    return np.ascontiguousarray(H[0, :, :N])


def combine_quarters(F) -> np.ndarray:
    """Eq. 16 and 22: f[y][x] = (F_v-[y][x] + F_v+[y][N-1-x]) + (F_h-[x][y] + F_h+[x][N-1-y]).

    F holds the quarter images F_q[tau][u] in the order v-, v+, h-, h+.  The '+' quarters
    were stored flipped about N-1, hence the reversed index; the 'h' quarters are the
    transposed problem (Eq. 16), hence [x][y].
    """
    F = np.asarray(F)
    v = F[0] + F[1][:, ::-1]
    h = F[2].T + F[3].T[::-1, :]
    return v + h
