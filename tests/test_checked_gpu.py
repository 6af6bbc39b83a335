"""The checked build (-DPULDA_CHECKED: every index read from device data
bounds-checked in the kernels) runs the z-step paths, fold-in, the batched
form and the server bit-exactly and without raising a bounds error.  It runs in
a process of its own, bound to the checked library through PULDA_LIB."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_runs_clean():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03581_gb300 import build
    lib = build.build_checked()
    env = dict(os.environ, PULDA_LIB=lib)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_cases.py")], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=1200)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-4000:]
    assert "all cases passed" in out.stdout
