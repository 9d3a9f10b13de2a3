"""Ragged sizes through the bounds-checked build (needs a GPU).

librm_checked.so is the library compiled with -DRM_CHECKED: every guarded index
(output and workspace stores, staged tiles, per-energy ranges) is tested, and a
failure is recorded and skipped instead of performed, with no trap.  The sweeps
of tests/checked_runner.py (channel counts 1, 2, 3, 16, 127, 129; pole counts
that are not multiples of 32; 1 to 140 energies; a grouped run of uneven waves;
the allocation-free entry point) run against it in a child process, which loads
only that library, and must finish with no guard failure and with cross sections
within the usual tolerances of the oracle.
"""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_ragged_sizes_under_bounds_checks():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lib = os.path.join(os.path.dirname(HERE), "paper_1403_5524_gb300", "librm_checked.so")
    assert os.path.exists(lib), "librm_checked.so is built by paper_1403_5524_gb300.build"
    env = dict(os.environ, RM_LIBRARY="checked")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_runner.py")], env=env, capture_output=True,
                       text=True, timeout=900)
    print(r.stdout[-3000:])
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    assert "CHECKED OK" in r.stdout

