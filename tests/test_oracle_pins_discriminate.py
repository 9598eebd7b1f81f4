"""The oracle's pins are discriminating: each plausible mistake below, planted in a copy of
the oracle (on the CPU, never in the product), makes at least one oracle pin fail."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MISTAKES = [
    ("geometry.py", "c if q in (0, 2) else (N - 1) - c", "c"),                 # storage not flipped
    ("geometry.py", "return np.pi / 2 + s", "return np.pi / 2 - s"),          # wrong h+ angle
    ("geometry.py", "    w[0] *= 0.5\n", ""),                                  # end row not halved
    ("dyadic.py", "s = (tau + 1) // 2", "s = tau // 2"),                       # floor instead of ceil
    ("dyadic.py", "half + (tau + 1) // 2]", "half + tau // 2]"),               # wrong pattern
    ("dyadic.py", "h = F[2].T + F[3].T[::-1, :]", "h = F[2] + F[3].T[::-1, :]"),  # missing transpose
    ("linogram.py", "np.where(wrap, (M - 1) - m, m)", "m"),                    # no mirror past pi
    ("linogram.py", "np.minimum(np.floor(tk), K - 1)", "np.minimum(np.round(tk), K - 1)"),
    ("iir.py", "acc = acc - a[k - 1] * y[..., n + k]", "acc = acc - a[k - 1] * p[..., n + k]"),
    ("iir.py", "acc = acc + b[k] * p[..., n - k]", "acc = acc + b[k] * p[..., n - k - 1]"),
    ("ramp.py", "out[n == 0] = 0.25", "out[n == 0] = 0.5"),
    ("fbp.py", "return acc * (np.pi / K)", "return acc * (2 * np.pi / K)"),
    # adjoints
    ("adjoint.py", "s0[:, t:] = a0[:, :W - t]", "s0[:, t + 1:] = a0[:, :W - t - 1]"),  # shift
    ("adjoint.py", "new[0::2, t, :] = a0 + a1", "new[0::2, t, :] = a0"),       # dropped term
    ("adjoint.py", "np.where(wrap, (M - 1) - m, m).ravel()", "m.ravel()"),     # no mirror
    ("adjoint.py", "return np.stack([g, g[:, ::-1], g.T, g[::-1, :].T])",
     "return np.stack([g, g[:, ::-1], g, g[::-1, :].T])"),                    # missing transpose
    # CNN corrector
    ("cnn.py", "xp[:, dy:dy + H, dx:dx + W],\n                             optimize=True)\n    return out",
     "xp[:, 2 - dy:2 - dy + H, 2 - dx:2 - dx + W],\n                             optimize=True)\n    return out"),  # convolution, not correlation
    ("cnn.py", "gh = gin * (hin > 0.0)", "gh = gin"),                          # ReLU mask dropped
    ("cnn.py", "return x + h[0], cache", "return h[0], cache"),                 # no skip connection
    ("cnn.py", "u = (u + 0x7FFF + ((u >> 16) & 1))", "u = (u + 0x8000)"),      # ties away from even
    ("cnn.py", "                h = bf16(h)\n", ""),                            # activations not stored in bf16
    # algebraic reconstruction
    ("sirt.py", "f = f + lam * cinv * back_project(", "f = f + lam * back_project("),  # no C^-1
    ("sirt.py", "(b - hough_project(f))", "(hough_project(f) - b)"),             # residual sign
    ("sirt.py", "scale = 1.0 / (row_weights(N) * np.sqrt(1.0 + sigma * sigma))",
     "scale = 1.0 / row_weights(N)"),                                         # no path length
    # fast Radon transform
    ("radon.py", "* np.sqrt(1.0 + sigma * sigma)", ""),                         # no path length
    ("radon.py", "return 3, np.tan(theta - np.pi / 2)", "return 2, np.tan(theta - np.pi / 2)"),
]


@pytest.mark.parametrize("fname,old,new", MISTAKES)
def test_planted_mistake_is_caught(tmp_path, fname, old, new):
    for d in ("oracle", "phantoms", "tests", "paper_2007_06289_gb300"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("*.so", "_build", "__pycache__", "csrc"))
    path = tmp_path / "oracle" / fname
    src = path.read_text()
    assert old in src
    path.write_text(src.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu",
                        "-p", "no:cacheprovider", "tests/test_oracle_ramp.py",
                        "tests/test_oracle_iir.py", "tests/test_oracle_geometry.py",
                        "tests/test_oracle_linogram.py", "tests/test_oracle_dyadic.py",
                        "tests/test_oracle_fbp.py", "tests/test_oracle_adjoint.py",
                        "tests/test_oracle_cnn.py", "tests/test_oracle_sirt.py",
                        "tests/test_oracle_radon.py"],
                       cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, r.stdout[-2000:]
