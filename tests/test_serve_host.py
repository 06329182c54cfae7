"""Serving scheduler core on the host (no GPU): compiled from the library's
own header with g++ and run; every scenario prints "ok <name>"."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_scheduler_core(tmp_path):
    exe = tmp_path / "sched_harness"
    src = os.path.join(ROOT, "tests", "cpp", "sched_harness.cpp")
    inc = os.path.join(ROOT, "paper_2203_10670_gb300", "csrc")
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", inc, src, "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    for name in ("pool_basics", "admission_by_footprint", "slots_limit_inflight", "steps_round_robin_and_chunking",
                 "latency_and_percentiles", "randomized_invariants", "cancel_requests"):
        assert f"ok {name}" in out.stdout
