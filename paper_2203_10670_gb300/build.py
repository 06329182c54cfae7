"""Build libfcfs.so in-tree with nvcc for sm_103a (GB300).

Each .cu translation unit is compiled in parallel into _build/, then linked
into paper_2203_10670_gb300/libfcfs.so (CUDA runtime linked statically, no
torch dependency).  Rebuilds only what is older than its sources or headers.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfcfs.so")
SOURCES = ["fcfs_host.cu", "fcfs_fwd.cu", "fcfs_fwd_tma.cu", "fcfs_fwd_tma_f32.cu", "fcfs_fwd_tma_bf16.cu", "fcfs_fwd_tma_u8.cu", "fcfs_fwd_rs_f32.cu", "fcfs_fwd_rs_bf16.cu", "fcfs_fwd3d_tma.cu", "fcfs_fwd3d_rs.cu", "fcfs_bwd.cu", "fcfs_bwd_tma.cu", "fcfs_bwd_dx_rs.cu", "fcfs_bwd_dx3d_tma.cu", "fcfs_full2d.cu", "fcfs_fused.cu", "fcfs_fused_tc.cu", "fcfs_fused_bwd.cu", "fcfs_tune.cu", "fcfs_serve.cu", "fcfs_noalloc.cu", "fcfs_psk_f32.cu", "fcfs_psk_bf16.cu", "fcfs_psk_host.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _headers():
    hs = [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    hs += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return hs


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = _headers()
    flags = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "-I" + INCLUDE, "-I" + CSRC] + ARCH
    if os.environ.get("FCFS_PTXAS_VERBOSE"):
        flags += ["-Xptxas", "-v"]
    jobs = []
    objs = []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        if force or _stale(obj, [path] + headers):
            jobs.append([nvcc()] + flags + ["-c", path, "-o", obj])

    def run(cmd):
        p = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, p

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for cmd, p in ex.map(run, jobs):
            if verbose or p.returncode != 0:
                sys.stderr.write(" ".join(cmd) + "\n" + p.stdout + p.stderr)
            if p.returncode != 0:
                raise RuntimeError(f"nvcc failed for {cmd[-3]}")
    if force or _stale(LIB, objs):
        cmd = [nvcc()] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs + ["-ldl"]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            sys.stderr.write(p.stdout + p.stderr)
            raise RuntimeError("linking libfcfs.so failed")
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
