"""CUDA-graph captures.

* The differentiable layer: the forward, input gradient and weight gradients
  of the c3 layer (BF16, 5/4 learnable per-channel taps) captured in one graph
  replay bit for bit what the eager calls produce (every kernel is
  deterministic, the weight gradient included).
* The timed benchmark step itself (c2: 16x3x1080x1920, bicubic 2/3, bicubic
  4/3, nearest 3/2, tiles chosen by the autotuner, one graph), built by the
  same function bench.py times, replayed and checked against the FP64 oracle
  on sampled outputs plus the edge rows and columns, FP32 and BF16."""
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


@pytest.mark.parametrize("dtype", (torch.float32, torch.bfloat16))
def test_c2_benchmark_step_graph_matches_oracle(F, orc, dtype):
    import bench

    replay, x, outs, axes = bench.c2_step(F, inputs, torch.device("cuda", 0), dtype, 16, tune=True, graph=True)
    F.fcfs_clear_plans()  # the graph keeps the tuned launches; later tests use the default tiles
    for y in outs.values():
        y.fill_(float("nan"))
    replay()
    replay()  # a second replay overwrites the first with the same values
    torch.cuda.synchronize()
    assert F.fcfs_device_status(clear=True) == 0
    xh = x.double().cpu().numpy()
    scale = float(np.abs(xh).max())
    for name, (r, s), m in bench.OPS:
        y = outs[name]
        idx = bench.sample_idx(tuple(y.shape), 100_000, 13)
        want = orc.resize_at(xh, [dict(r=r, s=s, method=m)] * 2, idx)
        got = bench.gather(y, idx)
        if m == 0:  # nearest: an exact copy
            assert np.array_equal(got, want)
        else:
            assert np.abs(got - want).max() <= (2e-6 if dtype == torch.float32 else 1e-2) * scale
