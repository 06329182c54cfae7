"""The N > 1 path of bench.py on the CPU: replicas only (the layer has no exchange
step), so ranks meet only to time the job (max over ranks) and rank 0 reports.
world_size 2 over gloo, loopback rendezvous."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, secs, out):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slow = bench.slowest_rank(secs[rank], torch.device("cpu"))
        rate = bench.job_rate(world, 5, 1e9, slow)
        out.put((rank, slow, rate))
    finally:
        torch.distributed.destroy_process_group()


def test_slowest_rank_and_job_rate_gloo():
    world, port = 2, _free_port()
    secs = [0.25, 0.5]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank_main, args=(r, world, port, secs, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest replica's time; the job rate counts all replicas' units
    assert [r[1] for r in res] == [0.5, 0.5]
    assert all(abs(r[2] - 2 * 5 * 1e9 / 0.5 / 1e9) < 1e-9 for r in res)


def test_single_process_no_group():
    import bench

    assert bench.slowest_rank(0.3, torch.device("cpu")) == 0.3
    assert bench.job_rate(1, 4, 2e9, 2.0) == 4.0


def test_reference_arm_under_torchrun_two_ranks():
    # rank 0 alone times the oracle and prints one line; rank 1 exits 0 without work
    pytest.importorskip("numpy")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    p = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
