"""Adjoints (transposes) of the linear steps of the fast method, for gradients with respect
to the sinogram (the differentiable form of Sec. 3-4).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The fast reconstruction of one slice is linear in the sinogram p:
    f = H(L(F p)),
F the recursive ramp filter (Eq. 12-13), L the resampling into the linogram quarters
(Eq. 14-15), H the quarter back projections along dyadic patterns with the Eq. 22 sum.
Its adjoint maps an image-space gradient g to p-bar = F^T L^T H^T g:
* F^T = F.  The causal filter is the lower-triangular Toeplitz matrix of its impulse
  response; the anticausal filter (the same coefficients run from the other end, Eq. 12-13)
  is exactly its transpose when both start from zero state; their sum is symmetric.
* H^T.  Undoing the index maps of Eq. 22 gives each quarter's gradient G_q[tau][u]; the
  transpose of F[tau][u] = sum_i L[i][u + d_tau(i)] is
      L-bar[i][c] = sum_tau G[tau][c - d_tau(i)]
  (terms with c - d_tau(i) outside [0, N) absent).  ``fht_stages_adjoint`` evaluates it by
  the stage recursion of ``dyadic.fht_stages`` run backwards, each stage transposed:
      A_{k-1}[2b][t][u]   = A_k[b][2t][u] + A_k[b][2t+1][u]
      A_{k-1}[2b+1][t][v] = A_k[b][2t][v - t] + A_k[b][2t+1][v - t - 1]
  (indices below 0 read as zero), in the stated order of the two terms.
* L^T.  Each linogram sample is w_i times a bilinear combination of at most four sinogram
  bins; the transpose adds w_i times the same four weights into those bins.
"""
from __future__ import annotations

import numpy as np

from .dyadic import _log2, dyadic_pattern
from .geometry import quarter_angle, quarter_r, row_weights
from .iir import iir_filter


def quarter_gradients(g) -> np.ndarray:
    """Transpose of ``dyadic.combine_quarters`` (Eq. 16, 22): image gradient g[y][x] ->
    G[4][tau][u] with G_v- = g, G_v+[tau][u] = g[tau][N-1-u], G_h- = g^T,
    G_h+[tau][u] = g[N-1-u][tau]."""
    g = np.asarray(g)
    return np.stack([g, g[:, ::-1], g.T, g[::-1, :].T])


def pattern_backproject_adjoint(G, W: int) -> np.ndarray:
    """Brute-force transpose of ``dyadic.pattern_backproject`` for one quarter (float64):
    L-bar[i][c] = sum_tau G[tau][c - d_tau(i)], c in [0, W)."""
    G = np.asarray(G, dtype=np.float64)
    N = G.shape[0]
    n = _log2(N)
    out = np.zeros((N, W))
    rows = np.arange(N)
    for tau in range(N):
        d = dyadic_pattern(n, tau)                     # [i]
        cols = np.arange(N)[None, :] + d[:, None]      # [i][u] -> column u + d_tau(i)
        ok = cols < W
        np.add.at(out, (np.broadcast_to(rows[:, None], cols.shape)[ok], cols[ok]),
                  np.broadcast_to(G[tau][None, :], cols.shape)[ok])
    return out


def fht_stages_adjoint(G, W: int, dtype=np.float32) -> np.ndarray:
    """The transposed stage recursion of the module docstring in ``dtype`` (each stage
    result rounded to ``dtype``): G[tau][u] (tau, u in [0, N)) -> L-bar[i][c], c in [0, W)."""
    G = np.asarray(G, dtype=dtype)
    N = G.shape[0]
    n = _log2(N)
    A = np.zeros((1, N, W), dtype=dtype)               # [strip b][tau][u]
    A[0, :, :N] = G
    for k in range(n, 0, -1):
        h = 1 << (k - 1)
        new = np.zeros((A.shape[0] * 2, h, W), dtype=dtype)
        for t in range(h):
            a0 = A[:, 2 * t, :]
            a1 = A[:, 2 * t + 1, :]
            new[0::2, t, :] = a0 + a1
            s0 = np.zeros_like(a0)
            s1 = np.zeros_like(a1)
            s0[:, t:] = a0[:, :W - t]
            s1[:, t + 1:] = a1[:, :W - t - 1]
            new[1::2, t, :] = s0 + s1
        A = new
    return np.ascontiguousarray(A[:, 0, :])


def fht_backproject_adjoint(g, W: int | None = None, brute: bool = False) -> np.ndarray:
    """Transpose of the whole back projection (quarters + Eq. 22 sum) for one slice:
    g[N][N] -> L-bar[4][N][W] (W = 2N by default), float64 (brute force) or float32 (the
    transposed stage recursion per quarter, as the GPU runs it)."""
    g = np.asarray(g)
    N = g.shape[0]
    W = 2 * N if W is None else W
    G = quarter_gradients(g)
    if brute:
        return np.stack([pattern_backproject_adjoint(G[q], W) for q in range(4)])
    return np.stack([fht_stages_adjoint(G[q].astype(np.float32), W) for q in range(4)])


def _scatter_row_lerp(out, rows, m, val):
    """Transpose of linear interpolation along the detector (zero outside [0, M))."""
    M = out.shape[-1]
    j0 = np.floor(m)
    f = m - j0
    j0 = j0.astype(np.int64)
    for j, w in ((j0, 1.0 - f), (j0 + 1, f)):
        ok = (j >= 0) & (j < M)
        np.add.at(out, (rows[ok], j[ok]), (w * val)[ok])


def linogram_adjoint(lbar, N: int, K: int, M: int) -> np.ndarray:
    """Transpose of ``linogram.linogram`` (Eq. 14-15): L-bar[4][N][2N] -> p-bar[K][M]
    (float64), with the same angle wrap (second sample at angle 0, detector mirrored,
    between theta_{K-1} and pi)."""
    lbar = np.asarray(lbar, dtype=np.float64)
    out = np.zeros((K, M))
    i = np.broadcast_to(np.arange(N)[:, None], (N, 2 * N))
    c = np.broadcast_to(np.arange(2 * N)[None, :], (N, 2 * N))
    w = row_weights(N)[i]
    for q in range(4):
        sigma = i / (N - 1)
        theta = quarter_angle(q, sigma)
        r = quarter_r(q, sigma, c, N)
        tk = theta * K / np.pi
        k0 = np.minimum(np.floor(tk), K - 1)
        ft = tk - k0
        k0 = k0.astype(np.int64)
        m = r + (M - 1) / 2.0
        v = w * lbar[q]
        _scatter_row_lerp(out, k0.ravel(), m.ravel(), ((1.0 - ft) * v).ravel())
        k1 = k0 + 1
        wrap = k1 >= K
        _scatter_row_lerp(out, np.where(wrap, 0, k1).ravel(),
                          np.where(wrap, (M - 1) - m, m).ravel(), (ft * v).ravel())
    return out


def fast_fbp_adjoint(g, N: int, K: int, M: int, b, a) -> np.ndarray:
    """Adjoint of ``fbp.fast_fbp`` (float64): image gradient g[N][N] -> sinogram gradient
    [K][M] = F(L^T(H^T g)), F symmetric."""
    lbar = fht_backproject_adjoint(np.asarray(g, np.float64), 2 * N, brute=True)
    return iir_filter(linogram_adjoint(lbar, N, K, M), b, a)
