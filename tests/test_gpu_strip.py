"""GPU parity of the polyphase strip kernels on every compiled window shape.

By default the strip kernels take the input gradients that have no
register-blocked tile kernel (the 8192^2 bicubic 7/5 workload among them) and
compete in the forward tile search; with FCFS_STRIP_KERNELS=1 they take every
2D descriptor in their scope.  The policy is read once per process, so the
cases run in a child process (tests/strip_cases.py) with that setting: forward
and input gradient, FP32 and BF16, three paddings, fixed and learnable taps,
ragged sizes spanning several strips and bands, against the FP64 oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_strip_kernels_match_oracle_on_every_compiled_shape():
    env = dict(os.environ, FCFS_STRIP_KERNELS="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "strip_cases.py")], env=env,
                       capture_output=True, text=True, timeout=1200)
    assert p.returncode == 0, p.stdout[-3000:] + p.stderr[-3000:]
    assert "cases=42" in p.stdout
