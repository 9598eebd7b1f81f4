"""Fitting the recursive ramp-filter coefficients (paper Sec. 3, text after Eq. 13).

The causal filter y(n) = sum_{k<Mb} b_k p(n-k) - sum_{k=1..Q} a_k y(n-k) and its mirror
image, the anticausal filter with the same coefficients, together approximate the
band-limited ramp kernel h of Eq. 7; their summed frequency response is
    H(w) = 2 Re[ B(e^{2 pi i w}) / A(e^{2 pi i w}) ],   w in cycles per sample,
and the ideal response is |w| on |w| <= 1/2.

The paper fits the coefficients by minimising a mean-square error between impulse
responses with a simplex (Nelder-Mead) or Powell search, and leaves the weighting and the
fitting length open.  This module fixes them as follows:

* Loss.  The mean of (H(w)/w - 1)^2 over 512 frequencies spaced evenly in log w on
  [1/(4M), 1/2].  By Parseval a frequency-weighted error of the response is a weighted
  error of the impulse response.  The weighting is chosen because the reconstruction
  error of FBP is (H(w)/|w| - 1) times the image spectrum, and phantom spectra fall
  roughly as 1/w^2, which makes every octave equally important; the unweighted
  impulse-response error lets a third-order filter lose the low frequencies (a uniform
  disk of N = 256 then reconstructs to about 0.28 instead of 1).
* DC.  sum_k b_k = 0, so H(0) = 0 like the ideal ramp (sum of h(n) over n is 0).
* Stability.  The feedback polynomial A is parameterised by reflection coefficients
  k_i = 0.99999 tanh(x_i), so every trial filter is stable, and poles beyond radius
  0.9999 are penalised, so the float32 modal realisation keeps a margin to |z| = 1.
* Search.  Nelder-Mead over x; for each trial A the optimal b is linear least squares
  (variable projection).  Several deterministic starts; the best is kept.

Running this file rewrites the committed table ``iir_coeffs.json`` and the C include
``csrc/iir_table.inc`` that the library compiles in as its built-in coefficients;
``--windows`` rewrites ``iir_windows.json``, order-3 fits of the apodised ramps (Shepp-Logan,
cosine, Hamming, Hann) that callers pass to fbp_plan as explicit coefficients; ``--mse``
rewrites ``iir_coeffs_mse.json``, order-3 fits under the paper's own objective, the plain
mean-square error of the impulse response: by Parseval the mean of (H(w) - w)^2 over a
uniform grid on (0, 1/2], with the same constraints and search (``mse_coefficients``).
"""
from __future__ import annotations

import json
import math
import os
import sys

import numpy as np

ORDERS = (2, 3, 4, 5, 6)          # Q = Mb
SIZES = tuple(1 << e for e in range(1, 13))   # N = 2 .. 4096
DEFAULT_ORDER = 3                 # the paper's reconstructions use Q = Mb = 3 (Sec. 5)
KMAX = 0.99999                    # bound on the reflection coefficients
PMAX = 0.9999                     # poles beyond this radius are penalised
_HERE = os.path.dirname(os.path.abspath(__file__))


def detector_bins(N: int) -> int:
    return int(math.ceil(N * math.sqrt(2.0)))


def reflection_to_poly(k) -> np.ndarray:
    """Step-up recursion: reflection coefficients -> a_1..a_Q of A(z) = 1 + sum a_j z^-j."""
    a = np.zeros(0)
    for km in k:
        a = np.concatenate([a + km * a[::-1], [km]])
    return a


def poly_to_reflection(a) -> np.ndarray:
    """Step-down recursion, the inverse of ``reflection_to_poly``."""
    a = np.asarray(a, dtype=np.float64).copy()
    k = np.zeros(a.size)
    for m in range(a.size, 0, -1):
        km = a[m - 1]
        k[m - 1] = km
        a = (a[:m - 1] - km * a[:m - 1][::-1]) / (1.0 - km * km)
    return k


def _basis(a, Mb, w):
    z = np.exp(-2j * np.pi * w)
    A = np.ones_like(z)
    for j, aj in enumerate(a):
        A = A + aj * z ** (j + 1)
    return np.stack([2.0 * (z ** k / A).real for k in range(Mb)], axis=1)


# Other FBP filters through the same fit (the end of Sec. 3): the ramp apodised by a window
# W(w) on |w| <= 1/2; the fit then matches H(w) to |w| W(w), the loss being the mean of
# ((H(w) - w W(w)) / w)^2 on the same log-spaced grid.
WINDOWS = ("ram-lak", "shepp-logan", "cosine", "hamming", "hann")
WINDOW_SIZES = (256, 512, 1024, 2048)       # sizes of the committed windowed-filter table


def window(w, name: str = "ram-lak") -> np.ndarray:
    w = np.asarray(w, dtype=np.float64)
    if name == "ram-lak":
        return np.ones_like(w)
    if name == "shepp-logan":
        return np.sinc(w)                    # sin(pi w) / (pi w)
    if name == "cosine":
        return np.cos(np.pi * w)
    if name == "hamming":
        return 0.54 + 0.46 * np.cos(2.0 * np.pi * w)
    if name == "hann":
        return 0.5 + 0.5 * np.cos(2.0 * np.pi * w)
    raise ValueError(f"unknown window {name!r}")


def best_b(a, Mb, w, target=None, relative=True):
    """Least-squares b with sum(b) = 0 for the given feedback coefficients, matching H(w)/w
    to `target` (the window; 1 for the plain ramp); returns (b, loss).  relative=False
    matches H(w) to w target(w) instead (an unweighted response error)."""
    target = np.ones_like(w) if target is None else target
    Phi = _basis(a, Mb, w)
    scale = w[:, None] if relative else np.ones_like(w)[:, None]
    want = target if relative else w * target
    D = (Phi[:, :-1] - Phi[:, -1:]) / scale
    bp, *_ = np.linalg.lstsq(D, want, rcond=None)
    b = np.concatenate([bp, [-bp.sum()]])
    r = (Phi @ b) / scale[:, 0] - want
    return b, float(np.mean(r * r))


def fit_coefficients(M: int, order: int, starts: int = 6, seed: int = 7, window_name="ram-lak",
                     objective: str = "log"):
    """Fit Q = Mb = order for a detector of M bins.  Returns (b, a, loss).
    objective "log": (H(w)/w - 1)^2 on a log-spaced grid (the default table); "impulse":
    (H(w) - w)^2 on a uniform grid, i.e. the impulse-response mean-square error."""
    from scipy.optimize import minimize
    relative = objective == "log"
    if relative:
        w = np.geomspace(1.0 / (4 * M), 0.5, 512)
    elif objective == "impulse":
        w = (np.arange(2 * M) + 0.5) / (4.0 * M)          # uniform on (0, 1/2)
    else:
        raise ValueError(objective)
    target = window(w, window_name)

    def loss(x):
        a = reflection_to_poly(KMAX * np.tanh(x))
        excess = np.abs(np.roots(np.concatenate([[1.0], a]))).max() - PMAX
        return best_b(a, order, w, target, relative)[1] + (1e3 * excess if excess > 0 else 0.0)

    rng = np.random.default_rng(seed)
    best = None
    for s in range(starts):
        if s % 2 == 0:
            # real poles spread geometrically towards z = 1, one negative pole
            spread = np.geomspace(2.0 / M, 0.6, max(order - 1, 1)) * rng.uniform(0.5, 2.0, max(order - 1, 1))
            poles = np.concatenate([1.0 - spread, [-rng.uniform(0.1, 0.8)]])[:order]
            k0 = poly_to_reflection(np.poly(np.clip(poles, -0.99, 0.9999))[1:])
        else:
            k0 = rng.uniform(-0.95, 0.95, order)
        x0 = np.arctanh(np.clip(k0 / KMAX, -0.99999, 0.99999))
        res = minimize(loss, x0, method="Nelder-Mead",
                       options=dict(maxiter=4000 * order, maxfev=4000 * order,
                                    xatol=1e-10, fatol=1e-14, adaptive=True))
        res = minimize(loss, res.x, method="Nelder-Mead",
                       options=dict(maxiter=4000 * order, maxfev=4000 * order,
                                    xatol=1e-12, fatol=1e-16, adaptive=True))
        if best is None or res.fun < best.fun:
            best = res
    a = reflection_to_poly(KMAX * np.tanh(best.x))
    b, f = best_b(a, order, w, target, relative)
    return b, a, f


def write_table(table, json_path, inc_path):
    with open(json_path, "w") as fh:
        json.dump(table, fh, indent=1)
    lines = ["/* Built-in recursive ramp-filter coefficients, written by iir_fit.py. */",
             "/* {N, order, {b_0..b_{order-1}}, {a_1..a_order}} */"]
    for e in table["entries"]:
        b = ", ".join(repr(float(v)) for v in e["b"])
        a = ", ".join(repr(float(v)) for v in e["a"])
        lines.append(f"{{{e['N']}, {e['order']}, {{{b}}}, {{{a}}}}},")
    with open(inc_path, "w") as fh:
        fh.write("\n".join(lines) + "\n")


def load_table(path=None):
    with open(path or os.path.join(_HERE, "iir_coeffs.json")) as fh:
        return json.load(fh)


def coefficients(N: int, order: int = DEFAULT_ORDER, table=None):
    """(b, a) from the committed table for image size N and order Q = Mb."""
    table = table or load_table()
    for e in table["entries"]:
        if e["N"] == N and e["order"] == order:
            return np.array(e["b"]), np.array(e["a"])
    raise KeyError((N, order))


def window_coefficients(N: int, window_name: str, order: int = DEFAULT_ORDER, table=None):
    """(b, a) of the committed windowed-filter table (iir_windows.json); the plain ramp
    comes from the main table."""
    if window_name == "ram-lak":
        return coefficients(N, order)
    if table is None:
        with open(os.path.join(_HERE, "iir_windows.json")) as fh:
            table = json.load(fh)
    for e in table["entries"]:
        if e["N"] == N and e["order"] == order and e["window"] == window_name:
            return np.array(e["b"]), np.array(e["a"])
    raise KeyError((N, window_name, order))


def _fit_window_entry(job):
    N, window_name = job
    M = detector_bins(N)
    b, a, f = fit_coefficients(M, DEFAULT_ORDER, window_name=window_name)
    return dict(N=N, order=DEFAULT_ORDER, window=window_name, M=M, loss=f,
                b=list(map(float, b)), a=list(map(float, a)))


def fit_windows():
    """Rewrite iir_windows.json: order-3 fits of every non-trivial window for WINDOW_SIZES."""
    import multiprocessing as mp
    jobs = [(N, wn) for N in WINDOW_SIZES for wn in WINDOWS if wn != "ram-lak"]
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        entries = pool.map(_fit_window_entry, jobs)
    with open(os.path.join(_HERE, "iir_windows.json"), "w") as fh:
        json.dump(dict(loss="mean ((H(w) - w W(w)) / w)^2, w log-spaced on [1/(4M), 1/2]",
                       entries=entries), fh, indent=1)


def mse_coefficients(N: int, order: int = DEFAULT_ORDER):
    """(b, a) of the committed impulse-response-MSE table (iir_coeffs_mse.json)."""
    with open(os.path.join(_HERE, "iir_coeffs_mse.json")) as fh:
        table = json.load(fh)
    for e in table["entries"]:
        if e["N"] == N and e["order"] == order:
            return np.array(e["b"]), np.array(e["a"])
    raise KeyError((N, order))


def _fit_mse_entry(N):
    M = detector_bins(N)
    b, a, f = fit_coefficients(M, DEFAULT_ORDER, objective="impulse")
    return dict(N=N, order=DEFAULT_ORDER, M=M, loss=f, b=list(map(float, b)), a=list(map(float, a)))


def fit_mse():
    """Rewrite iir_coeffs_mse.json: order-3 impulse-response MSE fits for WINDOW_SIZES."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(len(WINDOW_SIZES), os.cpu_count() or 1)) as pool:
        entries = pool.map(_fit_mse_entry, WINDOW_SIZES)
    with open(os.path.join(_HERE, "iir_coeffs_mse.json"), "w") as fh:
        json.dump(dict(loss="mean (H(w) - w)^2, w uniform on (0, 1/2): the impulse-response MSE",
                       entries=entries), fh, indent=1)


def _fit_entry(job):
    N, order = job
    M = detector_bins(N)
    b, a, f = fit_coefficients(M, order)
    poles = np.abs(np.roots(np.concatenate([[1.0], a])))
    print(f"N={N} order={order} loss={f:.4g} max|pole|={poles.max():.6f}", flush=True)
    return dict(N=N, order=order, M=M, loss=f, b=list(map(float, b)), a=list(map(float, a)))


def main(argv):
    """Fit the sizes given on the command line (default: all) and merge them into the table."""
    import multiprocessing as mp
    sizes = [int(v) for v in argv[1:]] or list(SIZES)
    jobs = [(N, order) for N in sizes for order in ORDERS]
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        fitted = pool.map(_fit_entry, jobs)
    old = []
    if argv[1:] and os.path.exists(os.path.join(_HERE, "iir_coeffs.json")):
        old = [e for e in load_table()["entries"] if e["N"] not in sizes]
    entries = sorted(old + fitted, key=lambda e: (e["N"], e["order"]))
    table = dict(default_order=DEFAULT_ORDER, loss="mean (H(w)/w - 1)^2, w log-spaced on [1/(4M), 1/2]",
                 entries=entries)
    write_table(table, os.path.join(_HERE, "iir_coeffs.json"),
                os.path.join(_HERE, "csrc", "iir_table.inc"))


if __name__ == "__main__":
    if sys.argv[1:2] == ["--windows"]:
        fit_windows()
    elif sys.argv[1:2] == ["--mse"]:
        fit_mse()
    else:
        main(sys.argv)
