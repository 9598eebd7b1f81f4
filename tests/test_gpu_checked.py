"""The bounds-checked library (libfbp_checked.so): tests/checked_cases.py in a subprocess
with FBP_LIBRARY pointing at it -- small parity cases with every access range-checked and
the status word clear afterwards, then a rejected geometry row setting the status word."""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def test_checked_library_cases():
    from paper_2007_06289_gb300 import build
    path = build.build(bounds_check=True)
    env = dict(os.environ, FBP_LIBRARY=path)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join("tests", "checked_cases.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    # every case ran and passed: none skipped or deselected
    summary = r.stdout.strip().splitlines()[-1]
    assert re.match(r"^\d+ passed(, \d+ warnings?)? in ", summary), summary
