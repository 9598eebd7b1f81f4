"""Seeded synthetic inputs: random-ellipse phantoms and their parallel-beam sinograms.

This module is the one input generator that both the CUDA path's tests/bench and the
CPU oracle's tests use.  It holds none of the reconstruction method's arithmetic: it only
draws phantoms and evaluates the textbook closed-form Radon transform of an ellipse,
optionally with Poisson counting noise.

Geometry (shared convention of the whole project)
-------------------------------------------------
* The image is N x N pixels, indexed ``img[y][x]``; pixel centres sit at integer
  (x, y) in [0, N), the rotation centre is c0 = (N - 1) / 2.
* Normalised coordinates map [-1, 1]^2 onto the image: X = (x - c0) / (N/2),
  Y = (y - c0) / (N/2).  One normalised unit is N/2 pixels.
* The sinogram is ``sino[k][m]`` with angle theta_k = k*pi/K (k in [0, K)) and detector
  offset r_m = m - (M - 1)/2 pixels; sino[k][m] is the line integral of the density over
  the line {(x - c0) cos(theta) + (y - c0) sin(theta) = r}, in pixel length units.

Phantom recipe: ten ellipses, centres uniform in the disk of radius 0.8, semi-axes
uniform in [0.05, 0.5], rotation uniform in [0, pi), density uniform in [-0.5, 1.0].
These stand in for the Shepp-Logan and CATPHAN phantoms used in the paper's experiments
(Sec. 5), which are not available here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Ellipse", "random_ellipses", "ellipse_sinogram", "ellipse_image",
    "poisson_log_noise", "phantom_stack", "geometry_for", "ellipse_sinogram_torch",
    "phantom_stack_torch",
]


@dataclass(frozen=True)
class Ellipse:
    x0: float      # centre, normalised units
    y0: float
    a: float       # semi-axis along direction alpha, normalised units
    b: float       # semi-axis across it
    alpha: float   # rotation of the a-axis, radians
    rho: float     # density


def geometry_for(N: int) -> tuple[int, int]:
    """(K, M) used by the workloads: K = 1.5 N angles, M = ceil(N sqrt 2) bins."""
    return (3 * N) // 2, int(math.ceil(N * math.sqrt(2.0)))


def random_ellipses(seed: int, count: int = 10) -> list[Ellipse]:
    """Draw ``count`` ellipses with the recipe stated in the module docstring."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        rad = 0.8 * math.sqrt(rng.uniform())
        phi = rng.uniform(0.0, 2.0 * math.pi)
        a, b = rng.uniform(0.05, 0.5, size=2)
        alpha = rng.uniform(0.0, math.pi)
        rho = rng.uniform(-0.5, 1.0)
        out.append(Ellipse(rad * math.cos(phi), rad * math.sin(phi), float(a), float(b),
                           float(alpha), float(rho)))
    return out


def _norm_sinogram(ellipses, theta, R):
    """Closed-form Radon transform of a sum of ellipses in normalised units.

    For one ellipse: p(theta, R) = 2 rho a b sqrt(s^2 - t^2) / s^2 when |t| <= s, else 0,
    with s^2 = a^2 cos^2(theta - alpha) + b^2 sin^2(theta - alpha) and
    t = R - x0 cos(theta) - y0 sin(theta).
    """
    th = theta[:, None]
    out = np.zeros((theta.size, R.size), dtype=np.float64)
    for e in ellipses:
        s2 = (e.a * np.cos(th - e.alpha)) ** 2 + (e.b * np.sin(th - e.alpha)) ** 2
        t = R[None, :] - e.x0 * np.cos(th) - e.y0 * np.sin(th)
        inside = s2 - t * t
        out += np.where(inside > 0, 2.0 * e.rho * e.a * e.b * np.sqrt(np.maximum(inside, 0.0)) / s2, 0.0)
    return out


def ellipse_sinogram(ellipses, N: int, K: int, M: int, noise_i0: float | None = None,
                     noise_seed: int | None = None) -> np.ndarray:
    """Sinogram [K][M] in pixel units (float64), optionally with Poisson noise."""
    theta = np.arange(K, dtype=np.float64) * (math.pi / K)
    r_px = np.arange(M, dtype=np.float64) - (M - 1) / 2.0
    p_norm = _norm_sinogram(ellipses, theta, r_px / (N / 2.0))
    if noise_i0 is not None:
        p_norm = poisson_log_noise(p_norm, noise_i0, noise_seed)
    return p_norm * (N / 2.0)


def poisson_log_noise(p_norm: np.ndarray, i0: float, seed: int | None) -> np.ndarray:
    """Counts n ~ Poisson(I0 exp(-p)); returns -ln(max(n, 1) / I0)."""
    rng = np.random.default_rng(seed)
    counts = rng.poisson(i0 * np.exp(-p_norm))
    return -np.log(np.maximum(counts, 1) / i0)


def ellipse_image(ellipses, N: int) -> np.ndarray:
    """Point-sampled phantom density at the pixel centres, ``img[y][x]`` (float64)."""
    c0 = (N - 1) / 2.0
    X = (np.arange(N, dtype=np.float64) - c0) / (N / 2.0)
    Y = X[:, None]
    X = X[None, :]
    img = np.zeros((N, N))
    for e in ellipses:
        dx, dy = X - e.x0, Y - e.y0
        u = (dx * math.cos(e.alpha) + dy * math.sin(e.alpha)) / e.a
        v = (-dx * math.sin(e.alpha) + dy * math.cos(e.alpha)) / e.b
        img += np.where(u * u + v * v <= 1.0, e.rho, 0.0)
    return img


def phantom_stack(N: int, slices: int, base_seed: int, noise_i0: float | None = None,
                  dtype=np.float32) -> np.ndarray:
    """[slices][K][M] sinograms of independent phantoms; slice i uses seed base_seed + i."""
    K, M = geometry_for(N)
    out = np.empty((slices, K, M), dtype=dtype)
    for i in range(slices):
        ell = random_ellipses(base_seed + i)
        out[i] = ellipse_sinogram(ell, N, K, M, noise_i0, noise_seed=(base_seed + i) * 7919 + 1)
    return out


# ----------------------------------------------------------------------------------------
# Device-side generator for large stacks.  Same formula, evaluated with torch in float64
# on whatever device the caller names; noise comes from a seeded torch generator, so the
# values differ from the numpy path's noise but are reproducible for a given seed.
# ----------------------------------------------------------------------------------------
def ellipse_sinogram_torch(ellipses, N: int, K: int, M: int, device, noise_i0=None,
                           noise_seed=None):
    import torch
    theta = torch.arange(K, dtype=torch.float64, device=device) * (math.pi / K)
    R = (torch.arange(M, dtype=torch.float64, device=device) - (M - 1) / 2.0) / (N / 2.0)
    th = theta[:, None]
    p = torch.zeros((K, M), dtype=torch.float64, device=device)
    for e in ellipses:
        s2 = (e.a * torch.cos(th - e.alpha)) ** 2 + (e.b * torch.sin(th - e.alpha)) ** 2
        t = R[None, :] - e.x0 * torch.cos(th) - e.y0 * torch.sin(th)
        inside = s2 - t * t
        p += torch.where(inside > 0, 2.0 * e.rho * e.a * e.b * torch.sqrt(inside.clamp_min(0)) / s2,
                         torch.zeros((), dtype=torch.float64, device=device))
    if noise_i0 is not None:
        g = torch.Generator(device=device)
        g.manual_seed(int(noise_seed))
        counts = torch.poisson(noise_i0 * torch.exp(-p), generator=g)
        p = -torch.log(counts.clamp_min(1.0) / noise_i0)
    return p * (N / 2.0)


def phantom_stack_torch(N: int, slices: int, base_seed: int, device, noise_i0=None, K=None,
                        M=None):
    """float32 [slices][K][M] stack on ``device``; slice i uses seed base_seed + i.  K and M
    default to geometry_for(N)."""
    import torch
    K0, M0 = geometry_for(N)
    K = K0 if K is None else K
    M = M0 if M is None else M
    out = torch.empty((slices, K, M), dtype=torch.float32, device=device)
    for i in range(slices):
        ell = random_ellipses(base_seed + i)
        out[i] = ellipse_sinogram_torch(ell, N, K, M, device, noise_i0,
                                        noise_seed=(base_seed + i) * 7919 + 1).float()
    return out
