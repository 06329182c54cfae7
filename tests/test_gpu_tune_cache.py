"""The on-disk plan cache (FCFS_TUNE_CACHE): a plan chosen by fcfs_tune_forward
in one process is appended to the file and loaded by the next process on the
same kind of device, which then runs the tuned tiles without timing again
(and computes the same output).  Each step runs in a child process, since the
file is read once per process."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, torch
sys.path.insert(0, {root!r})
from paper_2203_10670_gb300 import build, fcfs, inputs
build.build()
x = inputs.uniform((2, 3, 200, 320), 5, device="cuda")
axes = [fcfs.Axis(4, 3, fcfs.BICUBIC)] * 2
before = fcfs.fcfs_plan_count()
if sys.argv[1] == "tune":
    y = torch.empty(fcfs.out_shape(x.shape, axes), device="cuda")
    d = fcfs.make_desc(x.shape, axes, 0, 0)
    fcfs.fcfs_tune_forward(d, x.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream, 2)
y = fcfs.resize(x, axes)
torch.save(y.cpu(), sys.argv[2])
print("plans", before, fcfs.fcfs_plan_count())
"""


def _run(mode, out, env):
    p = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT), mode, out], env=env, capture_output=True,
                       text=True, timeout=600)
    assert p.returncode == 0, p.stdout + p.stderr
    return [int(v) for v in p.stdout.split("plans")[-1].split()]


def test_plans_persist_across_processes(tmp_path):
    import torch

    cache = tmp_path / "plans.txt"
    env = dict(os.environ, FCFS_TUNE_CACHE=str(cache))
    b0, a0 = _run("tune", str(tmp_path / "y0.pt"), env)
    assert b0 == 0 and a0 >= 1
    lines = cache.read_text().splitlines()
    assert lines and all(line.startswith("fcfs-plan ") and len(line.split()) == 26 for line in lines)
    b1, a1 = _run("plain", str(tmp_path / "y1.pt"), env)
    assert b1 >= 1 and a1 == b1  # loaded from the file, nothing tuned here
    b2, _ = _run("plain", str(tmp_path / "y2.pt"), {k: v for k, v in os.environ.items() if k != "FCFS_TUNE_CACHE"})
    assert b2 == 0
    y0, y1, y2 = (torch.load(tmp_path / f"y{k}.pt") for k in range(3))
    assert torch.equal(y0, y1) and torch.equal(y1, y2)
