"""The bounds-checked debug build (TFLBM_CHECK_BOUNDS) on the tiny and ragged
lattices: every global and shared index the step kernels compute is checked
against its buffer; a bad one would set TF_LBM_STATUS_BOUNDS (and be
redirected to element 0) instead of trapping.  No index may be out of range,
and results must still match the oracle.  The checked library is loaded in a
child process, so it never mixes with the normal build of this process."""
import os
import subprocess
import sys

import pytest

pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bounds_checked_build_tiny_and_ragged_lattices():
    from paper_1810_07642_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, TFLBM_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_check_run.py")], env=env,
                       capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-4000:]
    assert "0 failures" in r.stdout
