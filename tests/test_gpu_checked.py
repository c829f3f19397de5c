"""The bounds-checked build (libsph_checked.so, -DSPH_CHECKED), in a process
of its own: parity on small cases with every list and permutation entry
tested before use, and a planted out-of-range candidate entry reported as
SPH_ERR_BOUNDS without any out-of-range access."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_parity_and_planted_bounds_error():
    env = dict(os.environ, SPH_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "_checked_run.py")], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "checked ok" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
