"""Pins of the (r, theta) -> (s, t) resampling (Sec. 4.2, Eq. 14-15)."""
import numpy as np
import pytest

from oracle import linogram, quarter_angle, row_weights

N, K, M = 16, 24, 23
RANGES = {0: (0.0, np.pi / 4), 1: (3 * np.pi / 4, np.pi), 2: (np.pi / 4, np.pi / 2),
          3: (np.pi / 2, 3 * np.pi / 4)}


def _true_r(q, i, c):
    """r of the quarter-q line (row i, stored column c) from its two end points, with the
    normal oriented so that its angle lies in the quarter's range."""
    c0 = (N - 1) / 2
    s = i / (N - 1)
    u = c if q in (0, 2) else N - 1 - c
    sign = -1.0 if q in (0, 2) else 1.0
    if q in (0, 1):
        p1, p2 = np.array([u, 0.0]), np.array([u + sign * s * (N - 1), N - 1.0])
    else:
        p1, p2 = np.array([0.0, u]), np.array([N - 1.0, u + sign * s * (N - 1)])
    d = (p2 - p1) / np.linalg.norm(p2 - p1)
    n = np.array([d[1], -d[0]])
    th = np.arctan2(n[1], n[0]) % (2 * np.pi)
    lo, hi = RANGES[q]
    if not (lo - 1e-12 <= th <= hi + 1e-12):
        n = -n
        th = np.arctan2(n[1], n[0]) % (2 * np.pi)
    assert lo - 1e-12 <= th <= hi + 1e-12 or abs(th - 2 * np.pi) < 1e-12
    return float(np.dot(p1 - c0, n))


def _no_wrap(q, i):
    tk = quarter_angle(q, i / (N - 1)) * K / np.pi
    return np.floor(tk) + 1 < K


def test_theta_independent_linear_in_r():
    alpha, beta = 0.37, -1.25
    r_m = np.arange(M) - (M - 1) / 2
    pt = np.tile(alpha * r_m + beta, (K, 1))
    L = linogram(pt, N)
    w = row_weights(N)
    checked = 0
    for q in range(4):
        for i in range(N):
            if not _no_wrap(q, i):
                continue
            for c in range(2 * N):
                r = _true_r(q, i, c)
                m = r + (M - 1) / 2
                if 0 <= m <= M - 1:
                    assert L[q, i, c] == pytest.approx(w[i] * (alpha * r + beta), abs=1e-12)
                    checked += 1
    assert checked > 1000


def test_angle_index_interpolation():
    pt = np.tile(np.arange(K, dtype=float)[:, None], (1, M))
    L = linogram(pt, N)
    w = row_weights(N)
    for q in range(4):
        for i in range(N):
            if not _no_wrap(q, i):
                continue
            tk = quarter_angle(q, i / (N - 1)) * K / np.pi
            c = N // 2 if q in (0, 2) else N // 2 - 1      # a column near the centre line
            assert L[q, i, c] == pytest.approx(w[i] * tk, abs=1e-12)


def test_wrap_past_last_angle_reads_mirrored_first_projection():
    # p(pi, r) = p(0, -r): v+ row 0 (sigma = 0) has theta = pi exactly.
    pt = np.zeros((K, M))
    pt[0] = np.arange(M) + 1.0
    L = linogram(pt, N)
    w0 = row_weights(N)[0]
    for c in range(N):
        r = _true_r(1, 0, c)
        m_mirror = (M - 1) / 2 - r
        assert L[1, 0, c] == pytest.approx(w0 * (m_mirror + 1.0), abs=1e-12)


def test_outside_detector_is_zero():
    pt = np.ones((K, M))
    L = linogram(pt, N)
    for q in range(4):
        for i in range(N):
            for c in range(2 * N):
                r = _true_r(q, i, c)
                if abs(r) > (M - 1) / 2 + 1:
                    assert L[q, i, c] == 0.0
