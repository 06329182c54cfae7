"""GPU parity of the fused FCFS + 1x1 mix + bias + activation kernels (the
tensor-core mix for up to 96 input channels, the CUDA-core mix above that, the
store epilogue without a mix) against the FP64 oracle's resize_fused (pinned on the CPU to the library construction plus
torch's float64 1x1 convolution and activations).

Bar per output channel o: |err| <= tol * (2 max|x| sum_c |mix[o][c]| + |bias[o]|)
with tol 1e-5 for FP32 results and 1e-2 for BF16 results (2 bounds the sum of
|weights| of one FCFS output, at most 1.25^2 for the Keys cubic; the
activations are 1-Lipschitz).
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


def _np(t):
    return t.double().cpu().numpy()


def check(F, orc, shape, ratios, method, pad, c_out, act, identity=False, bias=True, din=torch.float32,
          dout=torch.float32, learn=False, align=0, seed=0, pad_value=0.0):
    n, C = shape[:2]
    x = inputs.uint8_pixels(shape, seed) if din == torch.uint8 else inputs.normal(shape, seed, dtype=din)
    mix = None if identity else inputs.normal((c_out, C), seed + 1)
    b = inputs.normal((c_out,), seed + 2) if bias else None
    axes, oaxes = [], []
    g = torch.Generator().manual_seed(seed + 3)
    for r, s in ratios:
        if learn:
            W, K = F.fcfs_make_weights(BILINEAR, r, s, 0)
            w = torch.from_numpy(np.tile(W[None], (C, 1, 1))) + 0.1 * torch.randn((C,) + W.shape, generator=g)
            w = w.float().contiguous()
            axes.append(F.Axis(r, s, BILINEAR, K, w.cuda()))
            oaxes.append(dict(r=r, s=s, K=K, w=w.double().numpy()))
        else:
            axes.append(F.Axis(r, s, method))
            oaxes.append(dict(r=r, s=s, method=method))
    y = F.resize_fused(x.cuda(), axes, None if mix is None else mix.cuda(), None if b is None else b.cuda(), act,
                       alpha=0.2, lo=-0.5, hi=0.75, pad=pad, pad_value=pad_value, out_dtype=dout, align=align)
    torch.cuda.synchronize()
    if learn:
        z = orc.resize(_np(x), oaxes, pad=pad, pad_value=pad_value, polyphase=True)
        v = z if mix is None else np.einsum("oc,nc...->no...", _np(mix), z)
        if b is not None:
            v = v + _np(b).reshape(1, -1, 1, 1)
        want = {0: v, 1: np.maximum(v, 0), 2: np.where(v >= 0, v, 0.2 * v), 3: np.clip(v, -0.5, 0.75)}[act]
    else:
        want = orc.resize_fused(_np(x), oaxes, None if mix is None else _np(mix), None if b is None else _np(b), act,
                                alpha=0.2, lo=-0.5, hi=0.75, pad=pad, pad_value=pad_value, align=align)
    got = _np(y)
    assert got.shape == want.shape
    mx = float(np.abs(_np(x)).max()) if x.numel() else 0.0
    mabs = np.ones((c_out, 1)) if mix is None else np.abs(_np(mix))
    scale = 2 * mx * mabs.sum(1) + (np.abs(_np(b)) if b is not None else 0)
    tol = (1e-5 if dout == torch.float32 else 1e-2) * scale.reshape(1, -1, 1, 1) + 1e-30
    bad = np.abs(got - want) > tol
    assert not bad.any(), f"{int(bad.sum())} outputs off; max err {float(np.abs(got - want).max()):.3e}"


@pytest.mark.parametrize("ratios,method", [(((2, 1), (2, 1)), BILINEAR), (((4, 3), (2, 3)), BICUBIC),
                                           (((3, 2), (5, 4)), NEAREST), (((1, 2), (2, 1)), BICUBIC)])
@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
@pytest.mark.parametrize("act", (0, 1, 2, 3))
def test_fused_mix_small(F, orc, ratios, method, pad, act):
    check(F, orc, (2, 3, 37, 71), ratios, method, pad, 5, act, pad_value=0.5, seed=act + 7 * method)


@pytest.mark.parametrize("c_in,c_out", [(16, 40), (8, 32), (5, 33), (64, 64), (96, 130), (100, 20)])
def test_fused_mix_many_channels(F, orc, c_in, c_out):
    check(F, orc, (2, c_in, 29, 50), ((2, 1), (2, 1)), BICUBIC, REFL, c_out, 1, seed=c_in)


@pytest.mark.parametrize("act", (0, 1, 3))
def test_fused_identity_epilogue(F, orc, act):
    check(F, orc, (2, 4, 33, 45), ((3, 2), (3, 2)), BICUBIC, REPL, 4, act, identity=True, seed=11 + act)
    check(F, orc, (1, 3, 20, 30), ((4, 3), (4, 3)), BILINEAR, CONST, 3, act, identity=True, bias=False,
          pad_value=0.5, seed=12)


def test_fused_dtypes_learnable_and_alignment(F, orc):
    check(F, orc, (2, 3, 37, 71), ((4, 3), (2, 3)), BICUBIC, REPL, 6, 1, din=torch.bfloat16, dout=torch.bfloat16)
    check(F, orc, (2, 3, 37, 71), ((2, 1), (2, 1)), BILINEAR, REFL, 6, 2, din=torch.bfloat16, dout=torch.float32)
    check(F, orc, (2, 3, 37, 71), ((3, 2), (3, 2)), BICUBIC, REPL, 4, 3, din=torch.uint8, dout=torch.float32)
    check(F, orc, (2, 3, 37, 71), ((5, 4), (5, 4)), BILINEAR, REFL, 7, 1, learn=True, seed=21)
    check(F, orc, (2, 3, 37, 71), ((4, 3), (2, 3)), BICUBIC, REPL, 5, 0, align=1, seed=22)


def test_fused_large_ratio_and_tiny_inputs(F, orc):
    check(F, orc, (1, 2, 5, 6), ((8, 1), (16, 1)), BILINEAR, REFL, 3, 1, seed=31)   # r_y r_x = 128
    for shape in ((1, 1, 1, 1), (1, 2, 2, 3), (2, 1, 3, 1)):
        check(F, orc, shape, ((3, 1), (2, 1)), BICUBIC, REPL, 2, 0, seed=32)


def test_fused_equals_resize_then_mix(F):
    """One kernel against two (the plain layer, then the channel mix as a library matmul)."""
    x = inputs.normal((2, 8, 64, 96), 41).cuda()
    mix = inputs.normal((12, 8), 42).cuda()
    b = inputs.normal((12,), 43).cuda()
    axes = [F.Axis(2, 1, BICUBIC)] * 2
    y = F.resize_fused(x, axes, mix, b, F.ACT_RELU)
    z = F.resize(x, axes)
    ref = torch.relu(torch.einsum("oc,nchw->nohw", mix.double(), z.double()) + b.double().view(1, -1, 1, 1))
    scale = 2 * float(x.abs().max()) * float(mix.abs().sum(1).max()) + float(b.abs().max())
    assert float((y.double() - ref).abs().max()) <= 1e-5 * scale


def test_fused_rejections(F):
    from paper_2203_10670_gb300._native import FCFSError

    x = torch.zeros(1, 3, 8, 8, device="cuda")
    with pytest.raises(FCFSError):  # r_y r_x = 1024 > 512
        F.resize_fused(x, [F.Axis(32, 1, BILINEAR), F.Axis(32, 1, BILINEAR)], torch.zeros(2, 3, device="cuda"))
    with pytest.raises(FCFSError):  # 3D
        F.resize_fused(torch.zeros(1, 3, 4, 4, 4, device="cuda"), [F.Axis(2, 1, BILINEAR)] * 3)
