"""Pins of the oracle's fused-layer gradients (y = act(mix FCFS(x) + bias), the
FCN layer of Sec. 1) against central finite differences of the oracle's own
fused forward, which is pinned elsewhere; CPU only.

Every term is checked: the input gradient, the mix and bias gradients and the
learnable taps' gradients, for each activation.  Points are drawn so that no
pre-activation lies within 1e-3 of a kink (where the derivative is a
convention, not a limit).  Without a mix, bias or activation the fused
gradient must reduce to the plain layer's input gradient.
"""
import numpy as np
import pytest

import oracle as orc

BILINEAR = orc.BILINEAR
REPL = orc.PAD_REPLICATE
ACTS = [(orc.ACT_NONE, {}), (orc.ACT_RELU, {}), (orc.ACT_LEAKY_RELU, {"alpha": 0.2}),
        (orc.ACT_CLAMP, {"lo": -0.4, "hi": 0.5})]


def _case(seed):
    rng = np.random.default_rng(seed)
    W, K = orc.make_weights(BILINEAR, 3, 2)
    axes = [dict(r=3, s=2, K=K, w=np.stack([W] * 3) + 0.05 * rng.standard_normal((3, 3, 2 * K + 1)))
            for _ in range(2)]
    x = rng.standard_normal((2, 3, 5, 6))
    mix = 0.5 * rng.standard_normal((4, 3))
    bias = 0.3 * rng.standard_normal(4)
    gy = rng.standard_normal((2, 4) + orc.out_shape(x.shape[2:], axes))
    return axes, x, mix, bias, gy


def _loss(x, axes, mix, bias, gy, act, kw):
    return float(np.vdot(orc.resize_fused(x, axes, mix, bias, act, **kw), gy))


def _kink_distance(x, axes, mix, bias, act, kw):
    z = orc.resize(x, axes, polyphase=True)
    v = np.einsum("oc,nc...->no...", mix, z) + bias.reshape(1, -1, 1, 1)
    if act in (orc.ACT_RELU, orc.ACT_LEAKY_RELU):
        return float(np.abs(v).min())
    if act == orc.ACT_CLAMP:
        return float(min(np.abs(v - kw["lo"]).min(), np.abs(v - kw["hi"]).min()))
    return np.inf


@pytest.mark.parametrize("act,kw", ACTS)
def test_fused_gradients_match_finite_differences(act, kw):
    for seed in range(40, 80):  # the first case with no pre-activation near a kink
        axes, x, mix, bias, gy = _case(seed)
        if _kink_distance(x, axes, mix, bias, act, kw) > 1e-3:
            break
    else:
        pytest.fail("no case away from the kinks")
    gx, gmix, gbias, gw = orc.resize_fused_backward(x, gy, axes, mix, bias, act, **kw)
    h = 1e-6
    rng = np.random.default_rng(3)

    def fd(perturb):
        lp = _loss(*perturb(+h), gy, act, kw)
        lm = _loss(*perturb(-h), gy, act, kw)
        return (lp - lm) / (2 * h)

    for _ in range(12):
        p = tuple(rng.integers(0, d) for d in x.shape)

        def px(e, p=p):
            x2 = x.copy()
            x2[p] += e
            return x2, axes, mix, bias
        assert abs(fd(px) - gx[p]) <= 1e-6 * max(1.0, abs(gx[p]))
    for o in range(mix.shape[0]):
        c = int(rng.integers(0, mix.shape[1]))

        def pm(e, o=o, c=c):
            m2 = mix.copy()
            m2[o, c] += e
            return x, axes, m2, bias

        def pb(e, o=o):
            b2 = bias.copy()
            b2[o] += e
            return x, axes, mix, b2
        assert abs(fd(pm) - gmix[o, c]) <= 1e-6 * max(1.0, abs(gmix[o, c]))
        assert abs(fd(pb) - gbias[o]) <= 1e-6 * max(1.0, abs(gbias[o]))
    for a in range(2):
        for _ in range(5):
            p = tuple(rng.integers(0, d) for d in axes[a]["w"].shape)

            def pw(e, a=a, p=p):
                ax2 = [dict(v) for v in axes]
                w = ax2[a]["w"].copy()
                w[p] += e
                ax2[a]["w"] = w
                return x, ax2, mix, bias
            assert abs(fd(pw) - gw[a][p]) <= 1e-6 * max(1.0, abs(gw[a][p]))


def test_reduces_to_the_plain_layer_gradient():
    axes, x, _, _, _ = _case(7)
    gy = np.random.default_rng(8).standard_normal((2, 3) + orc.out_shape(x.shape[2:], axes))
    gx, gmix, gbias, gw = orc.resize_fused_backward(x, gy, axes)
    assert gmix is None and gbias is None
    assert np.array_equal(gx, orc.adjoint_dx(gy, x.shape[2:], axes))
    for got, want in zip(gw, orc.weight_grad(x, gy, axes)):
        assert np.array_equal(got, want)


def test_derivative_conventions_at_the_kinks():
    v = np.array([-1.0, 0.0, 1.0, -0.4, 0.5])
    assert orc.act_derivative(v, orc.ACT_RELU).tolist() == [0, 0, 1, 0, 1]
    assert orc.act_derivative(v, orc.ACT_LEAKY_RELU, alpha=0.2).tolist() == [0.2, 0.2, 1, 0.2, 1]
    assert orc.act_derivative(v, orc.ACT_CLAMP, lo=-0.4, hi=0.5).tolist() == [0, 1, 0, 1, 1]
    assert orc.act_derivative(v, orc.ACT_NONE).tolist() == [1] * 5
