"""Out-of-bounds write checks with canary-padded buffers (the stand-in for a
memory checker, which this pool does not offer).

Every output buffer a kernel writes (forward outputs, input and weight
gradients, the non-separable layer's gradients, serving outputs placed by the
caller, the fused layer's output) is allocated inside a larger buffer whose
4 KiB before and after are filled with a NaN bit pattern.  After the call the
guard bytes must be untouched, and no element of the output itself may still
hold the pattern (outputs are fully overwritten).  Shapes are ragged so that
edge tiles, partial vectors and padding folds are exercised on every path:
bulk-copy, register-blocked and gather-staged kernels, 1D/2D/3D, FP32 and BF16.
"""
import numpy as np
import pytest
import torch

from paper_2203_10670_gb300 import inputs

pytestmark = pytest.mark.gpu

NEAREST, BILINEAR, BICUBIC = 0, 1, 2
GUARD = 4096  # bytes on each side
_BITS = {torch.float32: (torch.int32, 0x7FA5A5A5), torch.bfloat16: (torch.int16, 0x7FA5)}


@pytest.fixture(scope="module")
def F():
    from paper_2203_10670_gb300 import build

    build.build()
    from paper_2203_10670_gb300 import fcfs

    return fcfs


class Guarded:
    """An output of `shape` in the middle of a buffer with GUARD bytes of pattern on each side."""

    def __init__(self, shape, dtype):
        self.dtype = dtype
        self.n = int(np.prod(shape))
        self.pad = GUARD // torch.tensor([], dtype=dtype).element_size()
        self.buf = torch.empty(self.n + 2 * self.pad, dtype=dtype, device="cuda")
        ity, pat = _BITS[dtype]
        self.ity, self.pat = ity, pat
        self.buf.view(ity).fill_(pat)
        self.t = self.buf[self.pad:self.pad + self.n].view(shape)

    def check(self):
        torch.cuda.synchronize()
        bits = self.buf.view(self.ity)
        assert bool((bits[:self.pad] == self.pat).all()), "write before the output"
        assert bool((bits[self.pad + self.n:] == self.pat).all()), "write past the output"
        assert not bool((bits[self.pad:self.pad + self.n] == self.pat).any()), "output not fully written"


FWD_CASES = [
    # (shape, ratios, method, dtype) -- widths chosen for the bulk-copy path (rows of 16-byte multiples)
    # and for the gather path (odd widths)
    ((2, 3, 37, 64), ((4, 3), (4, 3)), BICUBIC, torch.float32),
    ((2, 3, 37, 64), ((2, 3), (2, 3)), BICUBIC, torch.bfloat16),
    ((1, 2, 41, 48), ((5, 4), (5, 4)), BILINEAR, torch.float32),
    ((3, 1, 29, 31), ((3, 2), (3, 2)), BILINEAR, torch.float32),
    ((1, 3, 33, 40), ((3, 2), (3, 2)), NEAREST, torch.float32),
    ((1, 3, 33, 41), ((3, 2), (3, 2)), NEAREST, torch.bfloat16),
    ((2, 2, 77), ((7, 5),), BICUBIC, torch.float32),
    ((1, 2, 13, 17, 32), ((3, 2), (3, 2), (3, 2)), BILINEAR, torch.float32),
    ((1, 1, 11, 14, 23), ((2, 3), (4, 3), (3, 2)), BICUBIC, torch.float32),
]


@pytest.mark.parametrize("shape,ratios,method,dtype", FWD_CASES)
@pytest.mark.parametrize("pad", (0, 1, 2))
def test_forward_writes_only_its_output(F, shape, ratios, method, dtype, pad):
    axes = [F.Axis(r, s, method) for r, s in ratios]
    x = inputs.uniform(shape, 3, device="cuda", dtype=dtype)
    out = Guarded(F.out_shape(shape, axes), dtype)
    F.resize(x, axes, pad, 0.5, out=out.t)
    out.check()


@pytest.mark.parametrize("shape,ratios,dtype", [
    ((2, 3, 37, 64), ((4, 3), (4, 3)), torch.float32),
    ((2, 3, 40, 64), ((2, 3), (2, 3)), torch.bfloat16),
    ((1, 2, 29, 31), ((5, 4), (7, 5)), torch.float32),
    ((1, 2, 13, 17, 32), ((3, 2), (3, 2), (3, 2)), torch.float32),
])
@pytest.mark.parametrize("pad", (0, 1, 2))
def test_input_gradient_writes_only_gx(F, shape, ratios, dtype, pad):
    axes = [F.Axis(r, s, BICUBIC) for r, s in ratios]
    gy = inputs.normal(F.out_shape(shape, axes), 4, device="cuda", dtype=dtype)
    gx = Guarded(shape, dtype)
    d = F.make_desc(shape, axes, F.FCFS_F32 if dtype == torch.float32 else F.FCFS_BF16,
                    F.FCFS_F32 if dtype == torch.float32 else F.FCFS_BF16, pad)
    F.fcfs_backward(d, None, gy.data_ptr(), gx.t.data_ptr(), None, None, 0, torch.cuda.current_stream().cuda_stream)
    gx.check()


@pytest.mark.parametrize("shape,ratio,K,dtype", [
    ((2, 4, 41, 64), (5, 4), 2, torch.float32),    # register-blocked weight gradient
    ((2, 4, 40, 64), (5, 4), 2, torch.bfloat16),
    ((1, 3, 23, 31), (3, 2), 2, torch.float32),    # gather-staged kernels
])
def test_weight_gradient_writes_only_gw(F, shape, ratio, K, dtype):
    C = shape[1]
    g = torch.Generator().manual_seed(5)
    ws_ = [torch.randn((C, ratio[0], 2 * K + 1), generator=g).cuda() for _ in range(2)]
    axes = [F.Axis(*ratio, BILINEAR, K, w) for w in ws_]
    x = inputs.normal(shape, 6, device="cuda", dtype=dtype)
    gy = inputs.normal(F.out_shape(shape, axes), 7, device="cuda", dtype=dtype)
    code = F.FCFS_F32 if dtype == torch.float32 else F.FCFS_BF16
    d = F.make_desc(shape, axes, code, code)
    gx = Guarded(shape, dtype)
    gws = [Guarded(tuple(w.shape), torch.float32) for w in ws_]
    nbytes = F.fcfs_backward_workspace(d)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    F.fcfs_backward(d, x.data_ptr(), gy.data_ptr(), gx.t.data_ptr(), [gw.t.data_ptr() for gw in gws],
                    ws.data_ptr(), nbytes, torch.cuda.current_stream().cuda_stream)
    gx.check()
    for gw in gws:
        gw.check()


def test_nonseparable_layer_writes_only_its_outputs(F):
    C = 3
    g = torch.Generator().manual_seed(8)
    w2d = torch.randn((C, 5, 5, 5, 5), generator=g).cuda()
    axes = [F.Axis(5, 4, BILINEAR), F.Axis(5, 4, BILINEAR)]
    shape = (2, C, 29, 37)
    x = inputs.normal(shape, 9, device="cuda")
    y = Guarded(F.out_shape(shape, axes), torch.float32)
    F.resize_full2d(x, axes, w2d, out=y.t)
    y.check()
    gy = inputs.normal(F.out_shape(shape, axes), 10, device="cuda")
    d = F.make_desc_full2d(shape, axes, w2d, F.FCFS_F32, F.FCFS_F32)
    gx = Guarded(shape, torch.float32)
    gw = Guarded(tuple(w2d.shape), torch.float32)
    nbytes = F.fcfs_backward_workspace(d)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    F.fcfs_backward(d, x.data_ptr(), gy.data_ptr(), gx.t.data_ptr(), [gw.t.data_ptr(), None], ws.data_ptr(), nbytes,
                    torch.cuda.current_stream().cuda_stream)
    gx.check()
    gw.check()


@pytest.mark.parametrize("dtype", (torch.float32, torch.bfloat16))
def test_fused_layer_writes_only_its_output(F, dtype):
    shape = (2, 8, 30, 40)
    axes = [F.Axis(2, 1, BILINEAR)] * 2
    x = inputs.normal(shape, 11, device="cuda", dtype=dtype)
    mix = inputs.normal((5, 8), 12, device="cuda")
    b = inputs.normal((5,), 13, device="cuda")
    y = Guarded((2, 5, 60, 80), dtype)
    F.resize_fused(x, axes, mix, b, F.ACT_RELU, out=y.t)
    # relu makes zeros, not the pattern; every element is still written
    y.check()


@pytest.mark.parametrize("dtype", (torch.float32, torch.bfloat16))
def test_serving_writes_only_caller_outputs(F, dtype):
    rng = np.random.default_rng(14)
    outs = []
    with F.Server(64 << 20, out_dtype=dtype, max_inflight=8, tile_budget_per_step=16) as sv:
        for k in range(12):
            H, W = int(rng.integers(20, 90)), int(rng.integers(20, 90))
            r, s = [(1, 2), (2, 3), (3, 4), (4, 3), (3, 2), (5, 2)][k % 6]
            x = inputs.uint8_pixels((1, 3, H, W), 100 + k, device="cuda")
            y = Guarded(F.out_shape(x.shape, [F.Axis(r, s, k % 3)] * 2), dtype)
            sv.submit(x, (r, s), k % 3, y=y.t)
            outs.append(y)
        sv.drain(60_000)
    for y in outs:
        y.check()


def test_device_status_clean_after_canaries(F):
    assert F.fcfs_device_status(clear=True) == 0
