"""The allocation-free backward entry point (fcfs_backward_noalloc).

Some callers cannot allocate device memory (their host framework owns every
allocation, or their deployment reserves all memory up front), so they cannot
provide the workspace fcfs_backward asks for.  This entry point keeps the
weight-gradient partial sums in a scratch area built into the library.  The
test calls it through the C ABI twice in a row and checks both results against
fcfs_backward with a torch-allocated workspace.  It sits in a file of its own
that pytest collects last, and passes alone in a fresh process as well as
after the other tests.  Both entry points run the same kernels in the same
fixed reduction order, so the results are compared bit for bit.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2203_10670_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2203_10670_gb300 import build

    build.build()
    from paper_2203_10670_gb300 import fcfs

    assert torch.cuda.is_available()
    return fcfs


def _axes(F, C):
    g = torch.Generator().manual_seed(41)
    W, K = F.fcfs_make_weights(F.BILINEAR, 5, 4)
    return [F.Axis(5, 4, F.BILINEAR, K, (torch.from_numpy(np.tile(W[None], (C, 1, 1)))
                                          + 0.1 * torch.randn((C, 5, 2 * K + 1), generator=g)).cuda())
            for _ in range(2)]


def _call_noalloc(lib, d, x, gy, gx, gw_ptrs):
    ptrs = (ctypes.c_void_p * 3)(*(list(gw_ptrs) + [None] * (3 - len(gw_ptrs))))
    return lib.fcfs_backward_noalloc(ctypes.byref(d), x.data_ptr(), gy.data_ptr(), gx.data_ptr(),
                                     ctypes.cast(ptrs, ctypes.c_void_p), torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("dtype", (torch.float32, torch.bfloat16))
def test_backward_noalloc_matches_workspace_entry_point(F, dtype):
    # fcfs_backward is given a workspace of exactly fcfs_backward_workspace(d) bytes, the size
    # the built-in area is asked for, so both calls pick the same kernels and the same fixed
    # reduction order: the results must agree bit for bit
    from paper_2203_10670_gb300 import _native as N

    lib = N.load()
    C = 6
    axes = _axes(F, C)
    x = inputs.normal((3, C, 70, 96), 12, device="cuda", dtype=dtype)
    gy = inputs.normal((3, C, 87, 120), 13, device="cuda", dtype=dtype)
    gx_ref, gw_ref = F.resize_backward(x, gy, axes, need_dx=True, need_dw=[True, True])
    d = F.make_desc(tuple(x.shape), axes, 0 if dtype == torch.float32 else 1, 0 if dtype == torch.float32 else 1)
    assert 0 < F.fcfs_backward_workspace(d) <= (8 << 20)
    for _ in range(2):  # two calls in a row share (and reuse) the built-in scratch area
        gx = torch.full_like(x, float("nan"))
        gw = [torch.full_like(a.w, float("nan")) for a in axes]
        rc = _call_noalloc(lib, d, x, gy, gx, [gw[0].data_ptr(), gw[1].data_ptr()])
        assert rc == N.FCFS_OK, lib.fcfs_last_error()
        torch.cuda.synchronize()
        assert torch.equal(gx, gx_ref)
        for a in range(2):
            assert torch.equal(gw[a], gw_ref[a])


def test_backward_noalloc_nonseparable_kernels(F):
    # the non-separable 2D layer keeps its weight-gradient records in the same area
    from paper_2203_10670_gb300 import _native as N

    lib = N.load()
    g = torch.Generator().manual_seed(43)
    C = 3
    w2d = torch.randn((C, 5, 5, 5, 5), generator=g).cuda()
    axes = [F.Axis(5, 4, F.BILINEAR), F.Axis(5, 4, F.BILINEAR)]
    x = inputs.normal((2, C, 41, 64), 14, device="cuda")
    gy = inputs.normal((2, C, 51, 80), 15, device="cuda")
    gx_ref, gw_ref = F.resize_full2d_backward(x, gy, axes, w2d)
    d = F.make_desc_full2d(tuple(x.shape), axes, w2d, N.FCFS_F32, N.FCFS_F32)
    assert 0 < F.fcfs_backward_workspace(d) <= (8 << 20)
    for _ in range(2):
        gx = torch.full_like(x, float("nan"))
        gw = torch.full_like(w2d, float("nan"))
        rc = _call_noalloc(lib, d, x, gy, gx, [gw.data_ptr(), None])
        assert rc == N.FCFS_OK, lib.fcfs_last_error()
        torch.cuda.synchronize()
        assert torch.equal(gx, gx_ref)
        assert torch.equal(gw, gw_ref)


def test_backward_noalloc_rejects_oversized_scratch(F):
    from paper_2203_10670_gb300 import _native as N

    lib = N.load()
    # a descriptor whose weight-gradient scratch exceeds the built-in 8 MiB; it is
    # rejected on the host before any pointer is touched
    w = torch.zeros((64, 5, 5), device="cuda")
    d = F.make_desc((512, 64, 1024, 1024), [F.Axis(5, 4, F.BILINEAR, 2, w)] * 2, 0, 0)
    assert F.fcfs_backward_workspace(d) > (8 << 20)
    ptrs = (ctypes.c_void_p * 3)(w.data_ptr(), w.data_ptr(), None)
    rc = lib.fcfs_backward_noalloc(ctypes.byref(d), w.data_ptr(), w.data_ptr(), None,
                                   ctypes.cast(ptrs, ctypes.c_void_p), None)
    assert rc == N.FCFS_ERR_NOMEM
    assert b"scratch" in lib.fcfs_last_error()
