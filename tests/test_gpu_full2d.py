"""GPU parity of the non-separable 2D kernels (forward, input gradient, weight
gradient) against the FP64 oracle (resize_full2d / adjoint_full2d /
weight_grad_full2d), which the CPU tests pin to the pad + grouped strided
convolution + pixel-shuffle construction and its autograd gradients.

Bars, element by element, with B the same oracle applied to |inputs| and
|weights| (the sum of the magnitudes of the terms of each result):
FP32 results |err| <= 1e-5 B (forward, input gradient) and 2e-5 B (weight
gradient, whose per-CTA partial sums run over up to a few thousand windows);
results stored as BF16 |err| <= 1e-2 B.  Weight gradients of BF16 inputs use
the FP32 bar: BF16 values are exact in FP32 and the arithmetic is FP32.
"""
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


def _w2d(C, ratios, Ks, per_channel, seed):
    (ry, _), (rx, _) = ratios
    shape = (ry, rx, 2 * Ks[0] + 1, 2 * Ks[1] + 1)
    if per_channel:
        shape = (C,) + shape
    return inputs.normal(shape, seed)


def _oax(ratios, Ks):
    return [dict(r=r, s=s, K=K) for (r, s), K in zip(ratios, Ks)]


def _axes(F, ratios):
    return [F.Axis(r, s, BILINEAR) for r, s in ratios]


def _np(t):
    return t.double().cpu().numpy()


def check_forward(F, orc, x_shape, ratios, Ks, pad, per_channel=True, din=torch.float32, dout=torch.float32,
                  pad_value=0.0, seed=0):
    x = inputs.uint8_pixels(x_shape, seed) if din == torch.uint8 else inputs.normal(x_shape, seed, dtype=din)
    w = _w2d(x_shape[1], ratios, Ks, per_channel, seed + 1)
    y = F.resize_full2d(x.cuda(), _axes(F, ratios), w.cuda(), pad, pad_value, out_dtype=dout)
    torch.cuda.synchronize()
    want = orc.resize_full2d(_np(x), _oax(ratios, Ks), _np(w), pad=pad, pad_value=pad_value)
    bound = orc.resize_full2d(np.abs(_np(x)), _oax(ratios, Ks), np.abs(_np(w)), pad=pad, pad_value=abs(pad_value))
    got = _np(y)
    assert got.shape == want.shape
    tol = 1e-5 if dout == torch.float32 else 1e-2
    bad = np.abs(got - want) > tol * bound + 1e-30
    assert not bad.any(), f"{int(bad.sum())} outputs off; max err {float(np.abs(got - want).max()):.3e}"


def check_backward(F, orc, x_shape, ratios, Ks, pad, per_channel=True, dtype=torch.float32, pad_value=0.0, seed=0):
    x = inputs.normal(x_shape, seed, dtype=dtype)
    w = _w2d(x_shape[1], ratios, Ks, per_channel, seed + 1)
    g_shape = tuple(x_shape[:2]) + tuple((n * r) // s for n, (r, s) in zip(x_shape[2:], ratios))
    gy = inputs.normal(g_shape, seed + 2, dtype=dtype)
    gx, gw = F.resize_full2d_backward(x.cuda(), gy.cuda(), _axes(F, ratios), w.cuda(), pad, pad_value)
    torch.cuda.synchronize()
    ax = _oax(ratios, Ks)
    want_dx = orc.adjoint_full2d(_np(gy), x_shape[2:], ax, _np(w), pad=pad)
    bound_dx = orc.adjoint_full2d(np.abs(_np(gy)), x_shape[2:], ax, np.abs(_np(w)), pad=pad)
    got = _np(gx)
    tol = 1e-5 if dtype == torch.float32 else 1e-2
    bad = np.abs(got - want_dx) > tol * bound_dx + 1e-30
    assert not bad.any(), f"dx: {int(bad.sum())} cells off; max err {float(np.abs(got - want_dx).max()):.3e}"
    want_dw = orc.weight_grad_full2d(_np(x), _np(gy), ax, per_channel, pad=pad, pad_value=pad_value)
    bound_dw = orc.weight_grad_full2d(np.abs(_np(x)), np.abs(_np(gy)), ax, per_channel, pad=pad,
                                      pad_value=abs(pad_value))
    got = _np(gw)
    assert got.shape == want_dw.shape
    bad = np.abs(got - want_dw) > 2e-5 * bound_dw + 1e-30
    assert not bad.any(), f"dW: {int(bad.sum())} entries off; max err {float(np.abs(got - want_dw).max()):.3e}"
    return gx, gw


RATIOS = [(((2, 1), (2, 1)), (1, 1)),   # bilinear x2 K_min
          (((2, 1), (2, 1)), (2, 2)),   # bicubic x2 K_min
          (((4, 3), (2, 3)), (3, 2)),   # anisotropic: 4/3 by 2/3, different T per axis
          (((3, 2), (1, 1)), (1, 2)),
          (((1, 2), (5, 4)), (1, 3)),
          (((2, 1), (1, 3)), (2, 2)),
          (((4, 4), (3, 1)), (2, 1))]   # E = 16 * 5 * 3 = 240 (one entry per thread)


@pytest.mark.parametrize("ratios,Ks", RATIOS)
@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
def test_forward(F, orc, ratios, Ks, pad):
    check_forward(F, orc, (2, 3, 37, 71), ratios, Ks, pad, pad_value=0.5 if pad == CONST else 0.0, seed=5)


@pytest.mark.parametrize("ratios,Ks", RATIOS)
@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
def test_backward(F, orc, ratios, Ks, pad):
    check_backward(F, orc, (2, 3, 37, 71), ratios, Ks, pad, pad_value=0.5 if pad == CONST else 0.0, seed=7)


@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
def test_shared_kernel(F, orc, pad):
    check_forward(F, orc, (3, 4, 29, 40), ((3, 2), (2, 1)), (2, 1), pad, per_channel=False, seed=11)
    check_backward(F, orc, (3, 4, 29, 40), ((3, 2), (2, 1)), (2, 1), pad, per_channel=False, seed=12)


@pytest.mark.parametrize("ratios,Ks", [(((4, 1), (4, 1)), (2, 2)),   # E = 400: several entries per thread
                                       (((8, 1), (8, 1)), (3, 3))])  # E = 3136, P = 64: smaller tiles
def test_many_entries(F, orc, ratios, Ks):
    check_forward(F, orc, (1, 2, 23, 45), ratios, Ks, REFL, seed=13)
    check_backward(F, orc, (1, 2, 23, 45), ratios, Ks, REFL, seed=14)


@pytest.mark.parametrize("shape", [(1, 2, 1, 1), (1, 1, 2, 3), (1, 1, 3, 2), (2, 1, 1, 5)])
@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
def test_tiny_inputs(F, orc, shape, pad):
    # virtual indices fold several times onto one or two real pixels
    check_forward(F, orc, shape, ((3, 1), (2, 1)), (3, 4), pad, seed=15)
    check_backward(F, orc, shape, ((3, 1), (2, 1)), (3, 4), pad, seed=16)


def test_bf16_and_u8(F, orc):
    check_forward(F, orc, (2, 3, 37, 71), ((4, 3), (2, 1)), (2, 2), REPL, din=torch.bfloat16, dout=torch.bfloat16)
    check_forward(F, orc, (2, 3, 37, 71), ((4, 3), (2, 1)), (2, 2), REFL, din=torch.bfloat16, dout=torch.float32)
    check_forward(F, orc, (2, 3, 37, 71), ((2, 1), (2, 1)), (2, 2), REPL, din=torch.uint8, dout=torch.float32)
    check_backward(F, orc, (2, 3, 37, 71), ((4, 3), (2, 1)), (2, 2), REFL, dtype=torch.bfloat16)


def test_larger_image_spans_many_tiles(F, orc):
    check_forward(F, orc, (1, 2, 130, 257), ((2, 1), (2, 1)), (2, 2), REPL, seed=21)
    check_backward(F, orc, (1, 2, 130, 257), ((2, 1), (2, 1)), (2, 2), REPL, seed=22)


def test_empty_output_gives_zero_gradients(F):
    x = torch.ones(1, 2, 1, 1, device="cuda")
    w = torch.ones(2, 1, 1, 3, 3, device="cuda")
    axes = [F.Axis(1, 2, BILINEAR), F.Axis(1, 2, BILINEAR)]
    y = F.resize_full2d(x, axes, w)
    assert y.shape == (1, 2, 0, 0)
    gx, gw = F.resize_full2d_backward(x, torch.empty(1, 2, 0, 0, device="cuda"), axes, w)
    assert float(gx.abs().sum()) == 0.0 and float(gw.abs().sum()) == 0.0


def test_outer_product_matches_separable(F):
    """w2d[c][jy][jx][my][mx] = wy[c][jy][my] wx[c][jx][mx] is the separable learnable layer."""
    C = 3
    wy = inputs.normal((C, 4, 7), 31).cuda()
    wx = inputs.normal((C, 2, 5), 32).cuda()
    w2d = torch.einsum("cam,cbn->cabmn", wy, wx).contiguous()
    x = inputs.normal((2, C, 50, 61), 33).cuda()
    ratios = ((4, 3), (2, 1))
    y2 = F.resize_full2d(x, _axes(F, ratios), w2d, REFL)
    ys = F.resize(x, [F.Axis(4, 3, BILINEAR, 3, wy), F.Axis(2, 1, BILINEAR, 2, wx)], REFL)
    torch.cuda.synchronize()
    scale = float(x.abs().max()) * float(wy.abs().sum(-1).max()) * float(wx.abs().sum(-1).max())
    assert float((y2 - ys).abs().max()) <= 2e-6 * scale


def test_weight_gradient_is_deterministic(F):
    x = inputs.normal((4, 3, 90, 120), 41).cuda()
    gy = inputs.normal((4, 3, 180, 240), 42).cuda()
    w = inputs.normal((3, 2, 2, 5, 5), 43).cuda()
    axes = _axes(F, ((2, 1), (2, 1)))
    a = F.resize_full2d_backward(x, gy, axes, w)
    b = F.resize_full2d_backward(x, gy, axes, w)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_module_autograd(F, orc):
    m = F.FCFSFull2d(3, ((2, 1), (4, 3)), method=BICUBIC).cuda()
    # the initial kernel is the outer product of the two axis tables: the fixed bicubic layer
    x = inputs.normal((2, 3, 33, 48), 51).cuda().requires_grad_(True)
    y = m(x)
    ref = F.resize(x.detach(), [F.Axis(2, 1, BICUBIC), F.Axis(4, 3, BICUBIC)])
    assert float((y.detach() - ref).abs().max()) <= 1e-5 * float(x.detach().abs().max())
    gy = inputs.normal(tuple(y.shape), 52).cuda()
    (y * gy).sum().backward()
    torch.cuda.synchronize()
    ax = [dict(r=2, s=1, K=m.axes[0].K), dict(r=4, s=3, K=m.axes[1].K)]
    w = _np(m.weight.detach())
    want_dx = orc.adjoint_full2d(_np(gy), (33, 48), ax, w)
    bound = orc.adjoint_full2d(np.abs(_np(gy)), (33, 48), ax, np.abs(w))
    assert (np.abs(_np(x.grad) - want_dx) <= 1e-5 * bound + 1e-30).all()
    want_dw = orc.weight_grad_full2d(_np(x.detach()), _np(gy), ax, True)
    bound = orc.weight_grad_full2d(np.abs(_np(x.detach())), np.abs(_np(gy)), ax, True)
    assert (np.abs(_np(m.weight.grad) - want_dw) <= 2e-5 * bound + 1e-30).all()


def test_rejections(F):
    from paper_2203_10670_gb300._native import FCFSError

    x = torch.zeros(1, 1, 8, 8, device="cuda")
    big = torch.zeros(8, 8, 9, 9, device="cuda")  # 64 * 81 = 5184 entries
    with pytest.raises(FCFSError):
        F.resize_full2d(x, _axes(F, ((8, 1), (8, 1))), big)
    w = torch.zeros(1, 2, 2, 3, 3, device="cuda")
    d = F.make_desc_full2d(x.shape, _axes(F, ((2, 1), (2, 1))), w, F.FCFS_F32, F.FCFS_F32)
    d.axis[0].w = w.data_ptr()  # per-axis weights and w2d together
    with pytest.raises(FCFSError):
        F.fcfs_forward(d, x.data_ptr(), x.data_ptr())


@pytest.mark.parametrize("pad", (REPL, REFL))
def test_forward_square_windows_compiled_taps(F, orc, pad):
    # the shapes with compile-time tap loops: 5 x 5 taps at x stride 4 (the 5/4 layer), 5 x 5 and 3 x 3 at stride 1
    check_forward(F, orc, (2, 3, 37, 71), ((5, 4), (5, 4)), (2, 2), pad, seed=9)
    check_forward(F, orc, (1, 2, 29, 43), ((2, 1), (3, 1)), (2, 2), pad, din=torch.bfloat16, dout=torch.bfloat16, seed=10)
    check_forward(F, orc, (1, 2, 29, 43), ((2, 1), (2, 1)), (1, 1), pad, seed=11)
