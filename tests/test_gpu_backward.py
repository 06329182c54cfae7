"""GPU parity of the backward kernels (input and weight gradients) against the
FP64 oracle's adjoint, which the CPU tests pin by the dot-product identity and
finite differences.

Bars: input gradient max|err| <= tol * max|g| * prod_a max_j sum_m |W_a| with
tol 2e-6 (FP32) / 1e-2 (BF16); weight gradient per tap
|err| <= 1e-5 (FP32) / 2e-2 (BF16) * sum of |summands| (the FP64 sum of
|g| * |x~| * prod of the other axes' |W|, computed by the oracle).
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


def _oaxes(axes):
    out = []
    for a in axes:
        d = dict(r=a.r, s=a.s, method=a.method, K=a.K)
        if a.w is not None:
            d["w"] = a.w.detach().double().cpu().numpy()
        out.append(d)
    return out


def _abs_axes(oaxes, orc):
    out = []
    for a in oaxes:
        b = dict(a)
        if "w" in a:
            b["w"] = np.abs(a["w"])
        else:
            W, K = orc.make_weights(a["method"], a["r"], a["s"], a.get("K", 0))
            b["w"], b["K"] = np.abs(W), K
        out.append(b)
    return out


def check_dx(F, orc, x_shape, axes, pad, dtype=torch.float32, seed=0):
    g_shape = tuple(x_shape[:2]) + tuple((n * a.r) // a.s for n, a in zip(x_shape[2:], axes))
    gy = inputs.normal(g_shape, seed, dtype=dtype)
    gx, _ = F.resize_backward(None, gy.cuda(), axes, pad, in_shape=x_shape, in_dtype=dtype, need_dx=True)
    torch.cuda.synchronize()
    assert F.fcfs_device_status(clear=True) == 0  # no bounded wait ran out, no plan invariant broken
    want = orc.adjoint_dx(gy.double().numpy(), x_shape[2:], _oaxes(axes), pad=pad)
    got = gx.double().cpu().numpy()
    scale = float(np.abs(gy.double().numpy()).max()) if gy.numel() else 1.0
    for a in _abs_axes(_oaxes(axes), orc):
        scale *= float(a["w"].sum(-1).max())
    tol = (2e-6 if dtype == torch.float32 else 1e-2) * max(scale, 1e-30)
    err = float(np.abs(got - want).max()) if got.size else 0.0
    assert err <= tol, f"dx max err {err:.3e} > {tol:.3e}"
    return err / max(scale, 1e-30)


@pytest.mark.parametrize("ratios", [((3, 2), (3, 2)), ((2, 3), (4, 3)), ((5, 4), (7, 5)), ((1, 2), (2, 1)),
                                    ((27, 11), (2, 11)), ((5, 2), (1, 1))])
@pytest.mark.parametrize("method", (NEAREST, BILINEAR, BICUBIC))
@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
def test_dx_fixed_methods(F, orc, ratios, method, pad):
    check_dx(F, orc, (2, 2, 45, 299), [F.Axis(r, s, method) for r, s in ratios], pad, seed=3 + method)


@pytest.mark.parametrize("ratio", ((2, 3), (4, 3), (3, 2)))
@pytest.mark.parametrize("method", (BILINEAR, BICUBIC))
@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
@pytest.mark.parametrize("dtype", (torch.float32, torch.bfloat16))
def test_dx_bulk_copy_same_ratio(F, orc, ratio, method, pad, dtype):
    # g rows of 16-byte multiples and the same ratio on both axes: the bulk-copy
    # input gradient, register-blocked where the adjoint span is compiled (x pass
    # with vector loads for r * sizeof = 8 or 16 bytes); 3 x 11 tiles, ragged
    W = 300 if ratio != (3, 2) else 304
    check_dx(F, orc, (2, 2, 263, W), [F.Axis(*ratio, method)] * 2, pad, dtype=dtype, seed=17 + method)


@pytest.mark.parametrize("ratio", ((3, 2), (2, 3), (7, 5)))
@pytest.mark.parametrize("pad", (REPL, REFL))
def test_dx_1d_and_tiny(F, orc, ratio, pad):
    check_dx(F, orc, (2, 3, 777), [F.Axis(*ratio, BICUBIC)], pad)
    for shape in ((1, 1, 1, 1), (1, 1, 2, 3), (1, 2, 5, 1), (1, 1, 3, 7)):
        check_dx(F, orc, shape, [F.Axis(*ratio, BILINEAR)] * 2, pad)


@pytest.mark.parametrize("ratios", [((3, 2),) * 3, ((2, 3), (4, 3), (5, 4))])
@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
@pytest.mark.parametrize("width", (37, 48))
def test_dx_3d(F, orc, ratios, pad, width):
    # width 48 gives g rows of 16-byte multiples (the bulk-copy volume kernel), 37 the gather kernel
    for method in (NEAREST, BILINEAR, BICUBIC):
        check_dx(F, orc, (1, 2, 17, 21, width), [F.Axis(r, s, method) for r, s in ratios], pad)


@pytest.mark.parametrize("ratios", [((3, 2),) * 3, ((2, 3), (4, 3), (5, 4)), ((1, 2), (3, 1), (2, 1))])
@pytest.mark.parametrize("pad", (REPL, REFL))
def test_dx_3d_bf16(F, orc, ratios, pad):
    check_dx(F, orc, (2, 2, 13, 18, 64), [F.Axis(r, s, BICUBIC) for r, s in ratios], pad, dtype=torch.bfloat16,
             seed=5)


@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
def test_dx_3d_tiny_and_many_tiles(F, orc, pad):
    for shape in ((1, 1, 1, 3, 8), (1, 1, 2, 1, 16), (1, 1, 3, 5, 8), (1, 1, 5, 2, 24)):
        for method in (BILINEAR, BICUBIC):
            check_dx(F, orc, shape, [F.Axis(3, 2, method)] * 3, pad)
    # depth chunks, ragged tiles on every axis, several tiles per CTA
    check_dx(F, orc, (3, 2, 41, 37, 136), [F.Axis(5, 4, BICUBIC), F.Axis(2, 3, BILINEAR), F.Axis(3, 2, BICUBIC)],
             pad, seed=9)


def test_dx_3d_learnable(F, orc):
    g = torch.Generator().manual_seed(12)
    axes = [F.Axis(r, s, BILINEAR, 2, (torch.randn((2, r, 5), generator=g) * 0.5).cuda())
            for r, s in ((3, 2), (5, 4), (3, 2))]
    check_dx(F, orc, (1, 2, 11, 13, 48), axes, REPL, seed=13)


def _learn_axes(F, C, ratios, K, per_channel, seed):
    g = torch.Generator().manual_seed(seed)
    axes = []
    for r, s in ratios:
        shape = (C, r, 2 * K + 1) if per_channel else (r, 2 * K + 1)
        axes.append(F.Axis(r, s, BILINEAR, K, (torch.randn(shape, generator=g) * 0.5).cuda()))
    return axes


def check_dw(F, orc, x, gy, axes, pad, pad_value=0.0, tol=1e-5):
    _, gws = F.resize_backward(x.cuda(), gy.cuda(), axes, pad, pad_value, need_dx=False,
                               need_dw=[a.w is not None for a in axes])
    torch.cuda.synchronize()
    oax = _oaxes(axes)
    want = orc.weight_grad(x.double().numpy(), gy.double().numpy(), oax, pad=pad, pad_value=pad_value)
    mag = orc.weight_grad(np.abs(x.double().numpy()), np.abs(gy.double().numpy()), _abs_axes(oax, orc), pad=pad,
                          pad_value=abs(pad_value))
    worst = 0.0
    for a, gw in enumerate(gws):
        if gw is None:
            continue
        got = gw.double().cpu().numpy()
        ratio = np.abs(got - want[a]) / np.maximum(mag[a], 1e-30)
        worst = max(worst, float(ratio.max()))
        assert (np.abs(got - want[a]) <= tol * mag[a] + 1e-30).all(), f"axis {a}: worst {float(ratio.max()):.2e}"
    return worst


@pytest.mark.parametrize("per_channel", (True, False))
@pytest.mark.parametrize("ratios,K", [(((5, 4), (5, 4)), 2), (((3, 2), (2, 3)), 3), (((7, 5), (4, 3)), 4)])
@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
def test_dw_and_dx_learnable(F, orc, per_channel, ratios, K, pad):
    C = 3
    axes = _learn_axes(F, C, ratios, K, per_channel, 17)
    x = inputs.normal((2, C, 41, 133), 5)
    gshape = (2, C) + tuple((n * r) // s for n, (r, s) in zip((41, 133), ratios))
    gy = inputs.normal(gshape, 6)
    check_dw(F, orc, x, gy, axes, pad, pad_value=0.3 if pad == CONST else 0.0)
    check_dx(F, orc, tuple(x.shape), axes, pad, seed=6)


@pytest.mark.parametrize("per_channel", (True, False))
@pytest.mark.parametrize("ratio,K", [((5, 4), 2), ((3, 2), 3), ((5, 4), 1), ((4, 3), 2), ((2, 3), 2)])
@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
def test_dw_register_blocked(F, orc, per_channel, ratio, K, pad):
    # learnable taps on both axes with one phase and tap count, 16-byte rows: the
    # register-blocked weight-gradient kernel (window per thread, all phases at once)
    C = 3
    axes = _learn_axes(F, C, (ratio, ratio), K, per_channel, 23)
    x = inputs.normal((2, C, 41, 144), 11)
    gshape = (2, C) + tuple((n * ratio[0]) // ratio[1] for n in (41, 144))
    gy = inputs.normal(gshape, 12)
    check_dw(F, orc, x, gy, axes, pad, pad_value=0.3 if pad == CONST else 0.0)


def test_dw_register_blocked_bf16(F, orc):
    axes = _learn_axes(F, 4, ((5, 4), (5, 4)), 2, True, 24)
    x = inputs.normal((2, 4, 37, 256), 13, dtype=torch.bfloat16)
    gy = inputs.normal((2, 4, 46, 320), 14, dtype=torch.bfloat16)
    check_dw(F, orc, x, gy, axes, REFL, tol=2e-2)


def test_dw_1d(F, orc):
    axes = _learn_axes(F, 4, ((5, 4),), 2, True, 4)
    x = inputs.normal((3, 4, 1001), 7)
    gy = inputs.normal((3, 4, 1251), 8)
    check_dw(F, orc, x, gy, axes, REPL)


def test_weight_gradient_is_deterministic(F):
    axes = _learn_axes(F, 8, ((5, 4), (5, 4)), 2, True, 5)
    x = inputs.normal((4, 8, 96, 96), 9).cuda()
    gy = inputs.normal((4, 8, 120, 120), 10).cuda()
    _, a = F.resize_backward(x, gy, axes, need_dx=False, need_dw=[True, True])
    _, b = F.resize_backward(x, gy, axes, need_dx=False, need_dw=[True, True])
    for u, v in zip(a, b):
        assert torch.equal(u, v)


def test_autograd_function_matches_oracle(F, orc):
    layer = F.FCFS(2, [(5, 4), (5, 4)], method=BILINEAR, learnable=True).cuda()
    x = inputs.normal((1, 2, 17, 23), 31).cuda().requires_grad_(True)
    y = layer(x)
    assert y.shape == (1, 2, 21, 28)
    g = inputs.normal(tuple(y.shape), 32).cuda()
    y.backward(g)
    oax = [dict(r=5, s=4, K=layer.Ks[a], w=layer.weights[a].detach().double().cpu().numpy()) for a in range(2)]
    want_dx = orc.adjoint_dx(g.double().cpu().numpy(), (17, 23), oax)
    want_dw = orc.weight_grad(x.detach().double().cpu().numpy(), g.double().cpu().numpy(), oax)
    assert np.abs(x.grad.double().cpu().numpy() - want_dx).max() <= 1e-5
    for a in range(2):
        assert np.abs(layer.weights[a].grad.double().cpu().numpy() - want_dw[a]).max() <= 1e-4


def test_config3_bf16_layer_full(F, orc):
    """8x64x256^2 bf16, 5/4, per-channel taps initialised to bilinear: forward,
    input and weight gradients against the oracle at full size."""
    shape = inputs.C3["shape"]
    C = shape[1]
    W, K = F.fcfs_make_weights(BILINEAR, 5, 4)
    axes = [F.Axis(5, 4, BILINEAR, K, torch.from_numpy(np.tile(W[None], (C, 1, 1))).cuda()) for _ in range(2)]
    x = inputs.normal(shape, inputs.C3["seed"], dtype=torch.bfloat16)
    y = F.resize(x.cuda(), axes)
    gy = inputs.normal(tuple(y.shape), inputs.C3["grad_seed"], dtype=torch.bfloat16)
    oax = _oaxes(axes)
    xo = x.double().numpy()
    want_y = orc.resize(xo, oax, polyphase=True)
    assert np.abs(y.double().cpu().numpy() - want_y).max() <= 1e-2 * float(np.abs(xo).max())
    gx, gws = F.resize_backward(x.cuda(), gy.cuda(), axes, need_dx=True, need_dw=[True, True])
    torch.cuda.synchronize()
    go = gy.double().numpy()
    want_dx = orc.adjoint_dx(go, shape[2:], oax)
    assert np.abs(gx.double().cpu().numpy() - want_dx).max() <= 1e-2 * float(np.abs(go).max())
    want_dw = orc.weight_grad(xo, go, oax)
    mag = orc.weight_grad(np.abs(xo), np.abs(go), _abs_axes(oax, orc))
    for a in range(2):
        err = np.abs(gws[a].double().cpu().numpy() - want_dw[a])
        assert (err <= 2e-2 * mag[a] + 1e-30).all()


def test_config5_backward_dx(F, orc):
    # 3D trilinear 3/2 input gradient at full size
    check_dx(F, orc, inputs.C5_3D["shape"], [F.Axis(3, 2, BILINEAR)] * 3, REPL, seed=77)


def test_config5_large_bicubic_7_5_dx_sampled(F, orc):
    """1x3x8192^2 bicubic 7/5 input gradient (the per-output gather kernel at this ratio) against the
    oracle's gather-form adjoint on 100,000 sampled input pixels plus the edge rows and columns."""
    shape = inputs.C5_2D["shape"]
    axes = [F.Axis(7, 5, BICUBIC)] * 2
    g_shape = tuple(shape[:2]) + tuple(n * 7 // 5 for n in shape[2:])
    gy = inputs.normal(g_shape, 78, device="cuda")
    gx, _ = F.resize_backward(None, gy, axes, in_shape=shape, in_dtype=torch.float32)
    torch.cuda.synchronize()
    assert F.fcfs_device_status(clear=True) == 0
    rng = np.random.default_rng(79)
    H, W = shape[2], shape[3]
    idx = list(rng.integers(0, int(np.prod(shape)), 100_000))
    for p in (0, shape[1] - 1):
        base = p * H * W
        idx += [base + c for c in range(0, W, 16)] + [base + (H - 1) * W + c for c in range(0, W, 16)]
        idx += [base + r * W for r in range(0, H, 16)] + [base + r * W + W - 1 for r in range(0, H, 16)]
    idx = np.array(idx, dtype=np.int64)
    go = gy.double().cpu().numpy()
    oax = _oaxes(axes)
    want = orc.adjoint_dx_at(go, shape[2:], oax, idx)
    got = gx.reshape(-1)[torch.from_numpy(idx).cuda()].double().cpu().numpy()
    scale = float(np.abs(go).max())
    for a in _abs_axes(oax, orc):
        scale *= float(a["w"].sum(-1).max())
    assert np.abs(got - want).max() <= 2e-6 * scale
