"""GPU parity of the fused layer's gradients (fcfs_backward_fused: the input,
mix, bias and learnable-tap gradients of y = act(mix FCFS(x) + bias)) against
the FP64 oracle's resize_fused_backward, which is pinned on the CPU to finite
differences of the fused forward.

Bars: each gradient element against tol times the sum of the magnitudes of
the terms that make it up (computed from the oracle's intermediates), with tol
1e-5 for FP32 data and 1e-2 when x or gy is BF16.  Cases are drawn so that no
pre-activation lies within 1e-5 of an activation kink (the FP32 and FP64
pre-activations differ by about 1e-7 of their size), where the two could take
the derivative on different sides.
"""
import numpy as np
import pytest
import torch

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


def _kink_distance(orc, v, act, lo, hi):
    if act in (orc.ACT_RELU, orc.ACT_LEAKY_RELU):
        return float(np.abs(v).min())
    if act == orc.ACT_CLAMP:
        return float(min(np.abs(v - lo).min(), np.abs(v - hi).min()))
    return np.inf


def run_case(F, orc, shape, ratio, method, pad, c_out, act, use_mix=True, use_bias=True, learn=False,
             dt=torch.float32, seed=0):
    n, c = shape[0], shape[1]
    alpha, lo, hi = 0.2, -0.3, 0.4
    for sd in range(seed, seed + 40):  # the first draw with no pre-activation near a kink
        rng = np.random.default_rng(sd)
        x = torch.from_numpy(rng.standard_normal(shape)).to(dt)
        mix = torch.from_numpy(0.5 * rng.standard_normal((c_out, c))).float() if use_mix else None
        b = torch.from_numpy(0.3 * rng.standard_normal(c_out)).float() if use_bias else None
        axes, oaxes = [], []
        for a in range(2):
            r, s = ratio[a]
            if learn:
                W, K = F.fcfs_make_weights(method, r, s)
                w = torch.from_numpy(np.stack([W] * c) + 0.05 * rng.standard_normal((c,) + W.shape)).float()
                axes.append(F.Axis(r, s, method, K, w.cuda()))
                oaxes.append(dict(r=r, s=s, K=K, w=w.double().numpy()))
            else:
                axes.append(F.Axis(r, s, method))
                oaxes.append(dict(r=r, s=s, method=method))
        xo = _np(x)
        z = orc.resize(xo, oaxes, pad=pad, polyphase=learn)
        v = z if mix is None else np.einsum("oc,nc...->no...", _np(mix), z)
        if b is not None:
            v = v + _np(b).reshape(1, -1, 1, 1)
        if _kink_distance(orc, v, act, lo, hi) > 1e-5:
            break
    else:
        pytest.fail("no draw away from the kinks")
    gy = torch.from_numpy(rng.standard_normal((n, c_out) + z.shape[2:])).to(dt)
    want = orc.resize_fused_backward(xo, _np(gy), oaxes, None if mix is None else _np(mix),
                                     None if b is None else _np(b), act, alpha, lo, hi, pad=pad)
    got = F.resize_fused_backward(x.cuda(), gy.cuda(), axes, None if mix is None else mix.cuda(),
                                  None if b is None else b.cuda(), act, alpha, lo, hi, pad=pad,
                                  need_dx=True, need_dmix=use_mix, need_dbias=use_bias, need_dw=[learn, learn])
    torch.cuda.synchronize()
    tol = 1e-5 if dt == torch.float32 else 1e-2
    # magnitude bounds of every gradient's terms, from the oracle's intermediates
    gv = _np(gy) * orc.act_derivative(v, act, alpha, lo, hi)
    # the same layer with every tap replaced by its magnitude
    absax = []
    for a in oaxes:
        W = a["w"] if learn else orc.make_weights(method, a["r"], a["s"])[0]
        absax.append(dict(r=a["r"], s=a["s"], K=(W.shape[-1] - 1) // 2, w=np.abs(W)))
    if mix is None:
        gz_abs = np.abs(gv)
    else:
        gz_abs = np.einsum("oc,no...->nc...", np.abs(_np(mix)), np.abs(gv))
    gx_bound = orc.adjoint_dx(gz_abs, xo.shape[2:], absax, pad=pad)
    gx = _np(got[0])
    assert (np.abs(gx - want[0]) <= tol * gx_bound + 1e-30).all()
    if use_mix:
        bound = np.einsum("nop,ncp->oc", np.abs(gv).reshape(n, c_out, -1), np.abs(z).reshape(n, c, -1))
        assert (np.abs(_np(got[1]) - want[1]) <= tol * bound + 1e-30).all()
    else:
        assert got[1] is None
    if use_bias:
        bound = np.abs(gv).sum(axis=(0, 2, 3))
        assert (np.abs(_np(got[2]) - want[2]) <= tol * bound + 1e-30).all()
    if learn:
        wb = orc.weight_grad(np.abs(xo), gz_abs, absax, pad=pad)
        for a in range(2):
            assert (np.abs(_np(got[3][a]) - want[3][a]) <= tol * wb[a] + 1e-7 * wb[a].max()).all()
    return got


@pytest.mark.parametrize("act", (0, 1, 2, 3))
def test_activations_fixed_bicubic(F, orc, act):
    run_case(F, orc, (2, 3, 19, 37), ((2, 1), (2, 1)), BICUBIC, REPL, 5, act, seed=10 * act)


@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
def test_pads_and_ratios(F, orc, pad):
    run_case(F, orc, (1, 4, 23, 29), ((3, 2), (4, 3)), BILINEAR, pad, 6, 1, seed=50 + pad)


def test_learnable_taps(F, orc):
    run_case(F, orc, (2, 3, 17, 21), ((5, 4), (5, 4)), BILINEAR, REPL, 4, 2, learn=True, seed=70)


def test_identity_and_no_bias(F, orc):
    run_case(F, orc, (2, 3, 16, 20), ((2, 1), (2, 1)), BICUBIC, REPL, 3, 1, use_mix=False, seed=80)
    run_case(F, orc, (2, 3, 16, 20), ((2, 1), (2, 1)), BICUBIC, REPL, 3, 3, use_bias=False, seed=81)


def test_bf16(F, orc):
    run_case(F, orc, (2, 8, 24, 40), ((2, 1), (2, 1)), BILINEAR, REPL, 8, 1, dt=torch.bfloat16, seed=90)


def test_wide_mix_several_tiles(F, orc):
    # 70 -> 66 channels: several 64 x 64 product tiles and a ragged tail in both channel counts
    run_case(F, orc, (1, 70, 12, 70), ((2, 1), (2, 1)), BILINEAR, REPL, 66, 0, seed=95)


def test_reproducible_and_rejections(F):
    rng = np.random.default_rng(3)
    x = torch.from_numpy(rng.standard_normal((2, 4, 32, 48))).float().cuda()
    mix = torch.from_numpy(rng.standard_normal((5, 4))).float().cuda()
    b = torch.zeros(5, device="cuda")
    axes = [F.Axis(2, 1, BICUBIC)] * 2
    gy = torch.randn((2, 5, 64, 96), device="cuda")
    a = F.resize_fused_backward(x, gy, axes, mix, b, 1, need_dmix=True, need_dbias=True)
    c = F.resize_fused_backward(x, gy, axes, mix, b, 1, need_dmix=True, need_dbias=True)
    for u, v in zip(a[:3], c[:3]):
        assert torch.equal(u, v)
    d = F.make_desc(x.shape, axes, F.FCFS_F32, F.FCFS_F32)
    e = F._fused_epilogue(4, mix, b, 1, 0.0, 0.0, 0.0)
    need = F.fcfs_backward_fused_workspace(d, e)
    assert need > 0
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    gx = torch.empty_like(x)
    with pytest.raises(F.FCFSError):  # workspace too small
        F.fcfs_backward_fused(d, e, x.data_ptr(), gy.data_ptr(), gx.data_ptr(), None, None, None, ws.data_ptr(),
                              need - 1)
    e2 = F._fused_epilogue(4, None, None, 1, 0.0, 0.0, 0.0)
    with pytest.raises(F.FCFSError):  # a mix gradient for a layer without a mix
        F.fcfs_backward_fused(d, e2, x.data_ptr(), torch.zeros(2, 4, 64, 96, device="cuda").data_ptr(),
                              gx.data_ptr(), mix.data_ptr(), None, None, ws.data_ptr(), need)


def test_module_autograd(F, orc):
    # FCFSFused trained through autograd: every parameter's gradient against the oracle
    torch.manual_seed(0)
    layer = F.FCFSFused(3, 4, [(2, 1), (3, 2)], BILINEAR, act=2, alpha=0.1, learnable=True).cuda()
    with torch.no_grad():
        layer.bias.copy_(torch.tensor([0.1, -0.2, 0.3, 0.05]))
        for w in layer.weights:
            w.add_(0.05 * torch.randn_like(w))
    x = torch.randn(2, 3, 14, 18, device="cuda", requires_grad=True)
    y = layer(x)
    gy = torch.randn_like(y)
    (y * gy).sum().backward()
    oaxes = [dict(r=r, s=s, K=k, w=w.detach().double().cpu().numpy())
             for (r, s), k, w in zip(layer.ratios, layer.Ks, layer.weights)]
    want = orc.resize_fused_backward(_np(x.detach()), _np(gy), oaxes, _np(layer.mix.detach()),
                                     _np(layer.bias.detach()), 2, 0.1)
    for got, w in ((x.grad, want[0]), (layer.mix.grad, want[1]), (layer.bias.grad, want[2]),
                   (layer.weights[0].grad, want[3][0]), (layer.weights[1].grad, want[3][1])):
        assert np.abs(_np(got) - w).max() <= 1e-4 * max(1.0, np.abs(w).max())
