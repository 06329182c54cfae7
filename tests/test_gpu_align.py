"""GPU parity of the sample-alignment variants (half-pixel centres, floor
nearest) and of the Keys parameter against the FP64 oracle, through the C ABI.
The oracle's variants are pinned to library interpolation on the CPU
(tests/test_oracle_pins.py).  Bars as for the paper's alignment: nearest
bit-exact, FP32 <= 2e-6 max|x| times the weights' absolute sums, BF16 <= 1e-2."""
import numpy as np
import pytest
import torch

from paper_2203_10670_gb300 import inputs

pytestmark = pytest.mark.gpu

NEAREST, BILINEAR, BICUBIC = 0, 1, 2
REPL, CONST, REFL = 0, 1, 2
PAPER, HALF, FLOOR = 0, 1, 2
TOL = {torch.float32: 2e-6, torch.bfloat16: 1e-2}


@pytest.fixture(scope="module")
def F():
    from paper_2203_10670_gb300 import build

    build.build()
    from paper_2203_10670_gb300 import fcfs

    return fcfs


def _oax(axes, align, cubic_a):
    return [dict(r=a.r, s=a.s, method=a.method, align=align, cubic_a=cubic_a) for a in axes]


def check(F, orc, x, axes, align, cubic_a=0.0, pad=REPL, pad_value=0.0):
    y = F.resize(x.cuda(), axes, pad, pad_value, align=align, cubic_a=cubic_a)
    torch.cuda.synchronize()
    want = orc.resize(x.double().numpy(), _oax(axes, align, cubic_a), pad=pad, pad_value=pad_value)
    got = y.double().cpu().numpy()
    assert got.shape == want.shape
    if got.size == 0:
        return
    if all(a.method == NEAREST for a in axes) and y.dtype == x.dtype:
        assert torch.equal(y.cpu(), torch.from_numpy(want).to(y.dtype)), "nearest must be bit-exact"
        return
    xmax = max(float(x.double().abs().max()), abs(pad_value) if pad == CONST else 0.0)
    err = float(np.abs(got - want).max()) / xmax
    assert err <= TOL[y.dtype] * 1.5 ** len(axes), f"{err:.3e}"


@pytest.mark.parametrize("align", (HALF, FLOOR))
@pytest.mark.parametrize("method", (NEAREST, BILINEAR, BICUBIC))
@pytest.mark.parametrize("ratio", [(3, 2), (2, 3), (4, 3), (5, 2), (1, 2), (2, 11), (27, 11)])
@pytest.mark.parametrize("width", (301, 304))
def test_2d_fp32(F, orc, align, method, ratio, width):
    # width 304 (16-byte rows) takes the bulk-copy kernels, 301 the gather kernels
    x = inputs.uniform((2, 3, 45, width), 101)
    for pad in (REPL, CONST, REFL):
        check(F, orc, x, [F.Axis(*ratio, method)] * 2, align, pad=pad, pad_value=-0.25)


@pytest.mark.parametrize("ratio", [(3, 2), (2, 3), (4, 3), (7, 5)])
@pytest.mark.parametrize("width", (77, 80))
def test_half_pixel_bicubic_keys_a075(F, orc, ratio, width):
    x = inputs.normal((1, 2, 33, width), 102)
    for pad in (REPL, REFL):
        check(F, orc, x, [F.Axis(*ratio, BICUBIC)] * 2, HALF, cubic_a=-0.75, pad=pad)
    # the Keys parameter also applies with the paper's alignment
    check(F, orc, x, [F.Axis(*ratio, BICUBIC)] * 2, PAPER, cubic_a=-0.75)


@pytest.mark.parametrize("align", (HALF, FLOOR))
def test_bf16_and_mixed_ratios(F, orc, align):
    x = inputs.normal((2, 2, 41, 128), 103, dtype=torch.bfloat16)
    for m in (NEAREST, BILINEAR, BICUBIC):
        check(F, orc, x, [F.Axis(3, 2, m), F.Axis(2, 3, m)], align, pad=REFL)


@pytest.mark.parametrize("align", (HALF, FLOOR))
@pytest.mark.parametrize("width", (41, 44))
def test_1d_and_3d(F, orc, align, width):
    for m in (NEAREST, BILINEAR, BICUBIC):
        check(F, orc, inputs.uniform((2, 3, 4 * width + 1), 104), [F.Axis(5, 4, m)], align, pad=REFL)
        check(F, orc, inputs.uniform((1, 2, 13, 17, width), 105), [F.Axis(3, 2, m), F.Axis(2, 3, m), F.Axis(4, 3, m)],
              align, pad=REPL)


def test_floor_nearest_s1_repeats(F):
    x = inputs.uniform((1, 2, 9, 12), 106).cuda()
    y = F.resize(x, [F.Axis(3, 1, NEAREST)] * 2, align=FLOOR)
    want = x.repeat_interleave(3, dim=2).repeat_interleave(3, dim=3)
    assert torch.equal(y, want)


def test_uint8_serving_path_half_pixel(F, orc):
    x = inputs.uint8_pixels((1, 3, 57, 96), 107).cuda()
    with F.Server(64 << 20, max_inflight=4, out_dtype=torch.float32, auto_release=False) as sv:
        rid = sv.submit(x, (4, 3), BILINEAR, align=HALF)
        sv.drain(60_000)
        y = sv.result(rid).clone()
        sv.release(rid)
    want = orc.resize(x.double().cpu().numpy(), [dict(r=4, s=3, method=BILINEAR, align=HALF)] * 2)
    assert np.abs(y.double().cpu().numpy() - want).max() <= 2e-6 * 255 * 1.5 ** 2


@pytest.mark.parametrize("align,cubic_a", [(HALF, 0.0), (HALF, -0.75), (FLOOR, 0.0)])
@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
@pytest.mark.parametrize("width", (37, 48))
def test_input_gradient(F, orc, align, cubic_a, pad, width):
    for ratios, method in ((((3, 2), (3, 2)), BICUBIC), (((2, 3), (4, 3)), BILINEAR), (((5, 4), (3, 2)), NEAREST)):
        axes = [F.Axis(r, s, method) for r, s in ratios]
        shape = (2, 2, 23, width)
        gshape = shape[:2] + tuple((n * r) // s for n, (r, s) in zip(shape[2:], ratios))
        gy = inputs.normal(gshape, 108)
        gx, _ = F.resize_backward(None, gy.cuda(), axes, pad, in_shape=shape, in_dtype=torch.float32, align=align,
                                  cubic_a=cubic_a)
        torch.cuda.synchronize()
        want = orc.adjoint_dx(gy.double().numpy(), shape[2:], _oax(axes, align, cubic_a), pad=pad)
        err = np.abs(gx.double().cpu().numpy() - want).max() / float(gy.abs().max())
        assert err <= 2e-6 * 1.5 ** 2 * 4, f"{ratios} {method}: {err:.3e}"


def test_input_gradient_3d_half_pixel(F, orc):
    axes = [F.Axis(3, 2, BILINEAR), F.Axis(2, 3, BICUBIC), F.Axis(4, 3, BILINEAR)]
    shape = (1, 2, 11, 13, 48)
    gshape = shape[:2] + tuple((n * a.r) // a.s for n, a in zip(shape[2:], axes))
    gy = inputs.normal(gshape, 109)
    gx, _ = F.resize_backward(None, gy.cuda(), axes, REFL, in_shape=shape, in_dtype=torch.float32, align=HALF)
    torch.cuda.synchronize()
    want = orc.adjoint_dx(gy.double().numpy(), shape[2:], _oax(axes, HALF, 0.0), pad=REFL)
    assert np.abs(gx.double().cpu().numpy() - want).max() <= 2e-6 * 1.5 ** 3 * 8 * float(gy.abs().max())
