"""Other FBP filters through the recursive fit (the end of Sec. 3): apodised ramps.

Pins: the oracle's closed-form impulse responses against numerical integration of the
ideal frequency responses; the committed windowed fits against those responses (their loss
recomputed here from the coefficients with independent code) and against the plain ramp
fit's quality; stability.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import ramp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def inverse_dtft(name, n):
    from scipy.integrate import quad
    return 2.0 * quad(lambda w: ramp.windowed_ramp_response(w, name) * np.cos(2 * np.pi * w * n),
                      0.0, 0.5, epsabs=1e-14, limit=200)[0]


@pytest.mark.parametrize("name,h", [("ram-lak", ramp.ramp_h), ("shepp-logan", ramp.shepp_logan_h),
                                    ("cosine", ramp.cosine_h)])
def test_closed_form_impulse_responses(name, h):
    for n in range(0, 9):
        assert abs(h(np.array([n]))[0] - inverse_dtft(name, n)) <= 1e-12


def test_shepp_logan_special_values():
    # h(0) = 2/pi^2, and the kernel sums to the response at w = 0, which is 0
    assert abs(ramp.shepp_logan_h(np.array([0]))[0] - 2 / np.pi ** 2) < 1e-15
    n = np.arange(-200000, 200001)
    assert abs(ramp.shepp_logan_h(n).sum()) < 1e-5


def test_windows_agree_with_the_fitting_code():
    from paper_2007_06289_gb300 import iir_fit
    w = np.linspace(0.0, 0.5, 101)
    for name in ramp.WINDOWS:
        np.testing.assert_allclose(iir_fit.window(w, name), ramp.window(w, name), rtol=0, atol=1e-15)


def response(b, a, w):
    """2 Re[B/A] on e^{2 pi i w}, from the coefficients (independent of the fitting code)."""
    z = np.exp(-2j * np.pi * w)
    B = sum(bk * z ** k for k, bk in enumerate(b))
    A = 1 + sum(ak * z ** (k + 1) for k, ak in enumerate(a))
    return 2 * (B / A).real


def test_committed_window_fits():
    with open(os.path.join(ROOT, "paper_2007_06289_gb300", "iir_windows.json")) as fh:
        table = json.load(fh)
    with open(os.path.join(ROOT, "paper_2007_06289_gb300", "iir_coeffs.json")) as fh:
        ramp_table = json.load(fh)
    names = {e["window"] for e in table["entries"]}
    assert names == set(ramp.WINDOWS) - {"ram-lak"}
    for e in table["entries"]:
        b, a = np.array(e["b"]), np.array(e["a"])
        M = e["M"]
        w = np.geomspace(1.0 / (4 * M), 0.5, 512)
        r = (response(b, a, w) - ramp.windowed_ramp_response(w, e["window"])) / w
        loss = float(np.mean(r * r))
        assert abs(loss - e["loss"]) <= 1e-9 * max(1.0, loss)
        ref = next(x for x in ramp_table["entries"] if x["N"] == e["N"] and x["order"] == e["order"])
        assert loss <= 1.3 * ref["loss"], (e["N"], e["window"], loss, ref["loss"])
        assert np.abs(np.roots(np.concatenate([[1.0], a]))).max() < 0.9999 + 1e-9
        assert abs(b.sum()) <= 1e-12 * np.abs(b).sum()
        # the response of the recursion itself (impulse response by the oracle's difference
        # equation, then its DTFT) is the same 2 Re[B/A]
        g = oracle.iir_impulse_response(b, a, 40 * M)
        n = np.arange(g.size)
        wm = w[::64]
        dtft = 2 * (g[None, :] * np.exp(-2j * np.pi * wm[:, None] * n[None, :])).sum(axis=1).real
        np.testing.assert_allclose(dtft, response(b, a, wm), rtol=0, atol=1e-6)


def _response(b, a, w):
    z = np.exp(-2j * np.pi * w)
    num = sum(bk * z ** k for k, bk in enumerate(b))
    den = 1.0 + sum(ak * z ** (k + 1) for k, ak in enumerate(a))
    return 2.0 * (num / den).real


def test_committed_impulse_mse_fits():
    # the paper's own objective (reading 20): mean (H(w) - w)^2 on a uniform grid, recomputed
    # here from the coefficients; stable, zero DC, and it trades the low frequencies away
    with open(os.path.join(ROOT, "paper_2007_06289_gb300", "iir_coeffs_mse.json")) as fh:
        table = json.load(fh)
    assert sorted(e["N"] for e in table["entries"]) == [256, 512, 1024, 2048]
    for e in table["entries"]:
        b, a, M = np.array(e["b"]), np.array(e["a"]), e["M"]
        assert np.abs(np.roots(np.concatenate([[1.0], a]))).max() < 1.0
        assert abs(b.sum()) <= 1e-12
        w = (np.arange(2 * M) + 0.5) / (4.0 * M)
        loss = float(np.mean((_response(b, a, w) - w) ** 2))
        assert abs(loss - e["loss"]) <= 1e-9 * max(1.0, loss)
        lo = w < 1.0 / M                                   # the lowest frequencies
        assert np.abs(_response(b, a, w[lo]) / w[lo] - 1).max() > 0.5


def test_committed_direct_fits_are_stable_and_zero_dc():
    with open(os.path.join(ROOT, "paper_2007_06289_gb300", "iir_direct_coeffs.json")) as fh:
        table = json.load(fh)
    have = {(e["N"], e["order"]) for e in table["entries"]}
    assert have == {(N, o) for N in (256, 512, 1024, 2048) for o in (3, 6)}
    for e in table["entries"]:
        b, a = np.array(e["b"]), np.array(e["a"])
        assert len(b) == e["order"] and len(a) == e["order"]
        assert np.abs(np.roots(np.concatenate([[1.0], a]))).max() < 0.99995
        assert abs(b.sum()) <= 1e-9 * np.abs(b).sum()
        assert e["loss"] <= e["loss_table"] * (1 + 1e-9)
        if e["source"] == "default table":
            from paper_2007_06289_gb300 import iir_fit
            b0, a0 = iir_fit.coefficients(e["N"], e["order"])
            assert np.array_equal(b, b0) and np.array_equal(a, a0)
