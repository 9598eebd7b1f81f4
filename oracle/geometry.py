"""The four line classes of the linogram and their (r, theta) parameters
(paper Sec. 4.1-4.2, Eq. 14-15).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Conventions (shared with the phantom generator): pixel centres at integer (x, y) in
[0, N), centre c0 = (N-1)/2, a sinogram line is {(x-c0) cos(theta) + (y-c0) sin(theta) = r}.

Readings fixed here:
* Quarter q and linogram row i hold lines of slope sigma_i = i/(N-1), i in [0, N):
    v-  : x = u - sigma y   (theta = atan(sigma),        in [0, pi/4])
    v+  : x = u + sigma y   (theta = pi - atan(sigma),   in [3pi/4, pi])
    h-  : y = u - sigma x   (theta = pi/2 - atan(sigma), in [pi/4, pi/2])
    h+  : y = u + sigma x   (theta = pi/2 + atan(sigma), in [pi/2, 3pi/4])
  which are the paper's classes L_v^-, L_v^+, L_h^-, L_h^+ with |t|/N = sigma (Sec. 4.1).
  The end rows sigma = 0 and sigma = 1 are shared by two classes; the row weights below
  halve them, so each direction is counted once.
* Stored column c holds intercept u = c for the '-' classes and u = N-1-c for the '+'
  classes (storage flipped about N-1), so that every class is back projected by the same
  positive-shift Hough transform.
* Back projection integrates over theta; with theta = atan(sigma) + const the Jacobian is
  d theta = d sigma / (1 + sigma^2) = d sigma / k_t^2 (k_t of Eq. 15).  Rows are weighted
  by the trapezoid rule in sigma: w_i = (1/(N-1)) / (1 + sigma_i^2), halved at i = 0 and
  i = N-1.  Over the four classes the weights approximate the integral over [0, pi).
"""
from __future__ import annotations

import numpy as np

QUARTERS = ("v-", "v+", "h-", "h+")


def slopes(N: int) -> np.ndarray:
    """sigma_i = i / (N-1) for i in [0, N)."""
    if N < 2:
        raise ValueError("N must be at least 2")
    return np.arange(N, dtype=np.float64) / (N - 1)


def quarter_angle(q: int, sigma) -> np.ndarray:
    """Normal angle theta of the quarter-q lines with slope sigma (table in the docstring)."""
    s = np.arctan(np.asarray(sigma, dtype=np.float64))
    if q == 0:
        return s
    if q == 1:
        return np.pi - s
    if q == 2:
        return np.pi / 2 - s
    if q == 3:
        return np.pi / 2 + s
    raise ValueError(q)


def intercept(q: int, c, N: int) -> np.ndarray:
    """Intercept u of stored column c (flipped storage for the '+' classes)."""
    c = np.asarray(c, dtype=np.float64)
    return c if q in (0, 2) else (N - 1) - c


def point_on_line(q: int, sigma, c, N: int):
    """One image point (x, y) on the quarter-q line of slope sigma stored at column c:
    (u, 0) for the mostly vertical classes, (0, u) for the mostly horizontal ones."""
    u = intercept(q, c, N)
    z = np.zeros(np.broadcast(np.asarray(sigma), u).shape)
    u = u + z
    return (u, z) if q in (0, 1) else (z, u)


def quarter_r(q: int, sigma, c, N: int) -> np.ndarray:
    """Signed distance r of the line from the image centre, measured along the normal of
    angle ``quarter_angle(q, sigma)``: r = (x - c0) cos(theta) + (y - c0) sin(theta) for a
    point (x, y) of the line."""
    c0 = (N - 1) / 2.0
    theta = quarter_angle(q, sigma)
    x, y = point_on_line(q, sigma, c, N)
    return (x - c0) * np.cos(theta) + (y - c0) * np.sin(theta)


def row_weights(N: int) -> np.ndarray:
    """Trapezoid weights w_i = (1/(N-1)) / (1 + sigma_i^2), halved at both ends."""
    s = slopes(N)
    w = (1.0 / (N - 1)) / (1.0 + s * s)
    w[0] *= 0.5
    w[-1] *= 0.5
    return w
