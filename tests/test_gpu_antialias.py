"""GPU parity of the antialiased downscale (descriptor field antialias = 1):
the fixed bilinear and bicubic kernels widened by s/r with renormalised
weights, against the FP64 oracle (itself pinned to float64 library
interpolation with antialias on padded inputs).  Forward 1D/2D/3D and the
input gradient, FP32 and BF16, every padding and both sample alignments; the
flag leaves upscales, nearest and learnable axes unchanged, and windows wider
than the kernel templates are refused on the host."""
import numpy as np
import pytest
import torch

from paper_2203_10670_gb300 import inputs

pytestmark = pytest.mark.gpu

NEAREST, BILINEAR, BICUBIC = 0, 1, 2
REPL, CONST, REFL = 0, 1, 2


@pytest.fixture(scope="module")
def F():
    from paper_2203_10670_gb300 import build

    build.build()
    from paper_2203_10670_gb300 import fcfs

    return fcfs


CASES = [(BILINEAR, (2, 3)), (BILINEAR, (1, 2)), (BILINEAR, (3, 7)), (BILINEAR, (2, 5)), (BILINEAR, (1, 4)),
         (BICUBIC, (2, 3)), (BICUBIC, (1, 2)), (BICUBIC, (3, 4))]


def _oax(axes, align):
    return [dict(r=a.r, s=a.s, method=a.method, align=align, antialias=1) for a in axes]


@pytest.mark.parametrize("method,ratio", CASES)
@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
@pytest.mark.parametrize("align", (0, 1))
def test_forward_2d(F, orc, method, ratio, pad, align):
    for dtype, shape in ((torch.float32, (2, 3, 61, 128)), (torch.bfloat16, (1, 2, 45, 77))):
        x = inputs.uniform(shape, 21, dtype=dtype)
        axes = [F.Axis(*ratio, method), F.Axis(*ratio, method)]
        y = F.resize(x.cuda(), axes, pad, 0.5, align=align, antialias=True)
        torch.cuda.synchronize()
        xh = x.double().numpy()
        want = orc.resize(xh, _oax(axes, align), pad=pad, pad_value=0.5)
        tol = 2e-6 if dtype == torch.float32 else 1e-2
        assert np.abs(y.double().cpu().numpy() - want).max() <= tol * max(1.0, float(np.abs(xh).max()))


@pytest.mark.parametrize("method,ratio", [(BILINEAR, (2, 3)), (BICUBIC, (1, 2)), (BILINEAR, (1, 4))])
def test_forward_1d_3d_and_mixed_axes(F, orc, method, ratio):
    x1 = inputs.uniform((2, 3, 301), 22)
    a1 = [F.Axis(*ratio, method)]
    y1 = F.resize(x1.cuda(), a1, antialias=True)
    w1 = orc.resize(x1.double().numpy(), _oax(a1, 0))
    assert np.abs(y1.double().cpu().numpy() - w1).max() <= 2e-6
    x3 = inputs.uniform((1, 2, 17, 23, 40), 23)
    a3 = [F.Axis(*ratio, method), F.Axis(3, 2, method), F.Axis(*ratio, method)]  # upscale axis unchanged
    y3 = F.resize(x3.cuda(), a3, REFL, antialias=True)
    w3 = orc.resize(x3.double().numpy(), _oax(a3, 0), pad=REFL)
    assert np.abs(y3.double().cpu().numpy() - w3).max() <= 2e-6


@pytest.mark.parametrize("method,ratio", CASES)
@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
def test_input_gradient(F, orc, method, ratio, pad):
    for dtype in (torch.float32, torch.bfloat16):
        shape = (2, 2, 53, 96)
        axes = [F.Axis(*ratio, method), F.Axis(*ratio, method)]
        gshape = tuple(shape[:2]) + tuple(n * ratio[0] // ratio[1] for n in shape[2:])
        gy = inputs.normal(gshape, 24, dtype=dtype)
        gx, _ = F.resize_backward(None, gy.cuda(), axes, pad, in_shape=shape, in_dtype=dtype, antialias=True)
        torch.cuda.synchronize()
        gh = gy.double().numpy()
        want = orc.adjoint_dx(gh, shape[2:], _oax(axes, 0), pad=pad)
        # every output's weights sum to one and are at most 1 in magnitude per tap: the bar is the
        # forward's, times the largest sum of |weights| a gradient entry collects (bounded by the
        # number of outputs a sample reaches on each axis, at most 2 R + 1 per axis)
        R = 1 if method == BILINEAR else 2
        bound = float(np.abs(gh).max()) * (2 * R + 1) ** 2
        tol = 2e-6 if dtype == torch.float32 else 1e-2
        assert np.abs(gx.double().cpu().numpy() - want).max() <= tol * bound


def test_flag_is_a_no_op_where_it_does_not_apply(F):
    x = inputs.uniform((1, 3, 40, 64), 25).cuda()
    for axes in ([F.Axis(4, 3, BICUBIC)] * 2, [F.Axis(3, 2, NEAREST)] * 2, [F.Axis(1, 2, NEAREST)] * 2,
                 [F.Axis(5, 5, BILINEAR)] * 2):
        assert torch.equal(F.resize(x, axes), F.resize(x, axes, antialias=True))
    W, K = F.fcfs_make_weights(BILINEAR, 1, 2)
    w = torch.from_numpy(W).cuda()
    learn = [F.Axis(1, 2, BILINEAR, K, w)] * 2
    assert torch.equal(F.resize(x, learn), F.resize(x, learn, antialias=True))


def test_too_wide_windows_are_refused(F):
    from paper_2203_10670_gb300 import _native as N

    x = inputs.uniform((1, 1, 40, 64), 26).cuda()
    with pytest.raises(F.FCFSError) as e:
        F.resize(x, [F.Axis(1, 4, BICUBIC)] * 2, antialias=True)  # 15 taps per phase
    assert e.value.status == N.FCFS_ERR_UNSUPPORTED
    with pytest.raises(F.FCFSError) as e:
        F.resize(x, [F.Axis(2, 11, BILINEAR)] * 2, antialias=True)  # 11 taps per phase
    assert e.value.status == N.FCFS_ERR_UNSUPPORTED


def test_device_status_clean(F):
    assert F.fcfs_device_status(clear=True) == 0
