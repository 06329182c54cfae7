"""CUDA-graph capture of the differentiable layer: the forward, input gradient
and weight gradients of the c3 layer (BF16, 5/4 learnable per-channel taps)
captured in one graph replay bit for bit what the eager calls produce (every
kernel is deterministic, the weight gradient included)."""
import numpy as np
import pytest
import torch

from paper_2203_10670_gb300 import inputs

pytestmark = pytest.mark.gpu

BILINEAR = 1


@pytest.fixture(scope="module")
def F():
    from paper_2203_10670_gb300 import build

    build.build()
    from paper_2203_10670_gb300 import fcfs

    return fcfs


def test_c3_forward_backward_in_one_graph(F):
    shape = (2, 64, 256, 256)
    W, K = F.fcfs_make_weights(BILINEAR, 5, 4)
    g = torch.Generator().manual_seed(5)
    wy = (torch.from_numpy(np.tile(W[None], (64, 1, 1))) + 0.05 * torch.randn((64,) + W.shape, generator=g)).float()
    wx = (torch.from_numpy(np.tile(W[None], (64, 1, 1))) + 0.05 * torch.randn((64,) + W.shape, generator=g)).float()
    ax = [F.Axis(5, 4, BILINEAR, K, wy.cuda().contiguous()), F.Axis(5, 4, BILINEAR, K, wx.cuda().contiguous())]
    x = inputs.normal(shape, 1, dtype=torch.bfloat16).cuda()
    oshape = F.out_shape(shape, ax)
    gy = inputs.normal(oshape, 2, dtype=torch.bfloat16).cuda()

    y_e = F.resize(x, ax)
    gx_e, gw_e = F.resize_backward(x, gy, ax, need_dx=True, need_dw=[True, True])
    torch.cuda.synchronize()

    d = F.make_desc(shape, ax, F.FCFS_BF16, F.FCFS_BF16)
    ws_bytes = F.fcfs_backward_workspace(d)
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device="cuda")
    y = torch.empty_like(y_e)
    gx = torch.empty_like(x)
    gw = [torch.empty_like(a.w) for a in ax]

    def step():
        st = torch.cuda.current_stream().cuda_stream
        F.fcfs_forward(d, x.data_ptr(), y.data_ptr(), st)
        F.fcfs_backward(d, x.data_ptr(), gy.data_ptr(), gx.data_ptr(), [w.data_ptr() for w in gw], ws.data_ptr(),
                        ws_bytes, st)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()  # eager warm-up on the capture stream
    side.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        step()
    for t in (y, gx, *gw):
        t.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, y_e)
    assert torch.equal(gx, gx_e)
    for a, b in zip(gw, gw_e):
        assert torch.equal(a, b)
    assert F.fcfs_device_status(clear=True) == 0
