"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test ties the oracle to a fact the paper or mathematics fixes:
  * the weight examples printed in Sec. 5.2 (golden fixture),
  * closed-form properties of the bilinear and Keys (a = -1/2) kernels,
  * exact-rational brute force of linear and Catmull-Rom interpolation,
  * the paper's own construction (pad -> strided conv -> pixelshuffle, Sec. 3.1
    and Sec. 4) composed from PyTorch CPU library ops in float64,
  * scipy's linear interpolation at the same sample positions,
  * invariants (constants, ramps, identity, unreduced ratios, separability),
  * adjoint identities and finite differences for the gradients.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

NEAREST, BILINEAR, BICUBIC = 0, 1, 2
REPL, CONST, REFL = 0, 1, 2
METHODS = (NEAREST, BILINEAR, BICUBIC)
# ratios of the workloads, the paper's extreme examples (Sec. 6: 2/11, 27/11) and simple ones
RATIOS = [(3, 2), (2, 3), (4, 3), (5, 4), (7, 5), (1, 1), (2, 1), (3, 1), (1, 2), (3, 4), (5, 2),
          (2, 11), (27, 11)]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_sec5_weights_3_2.json")


# --------------------------------------------------------------- kernels (P3)

def test_keys_kernel_interpolates(orc):
    assert orc.kernel(BICUBIC, 0.0) == 1.0
    for t in (1.0, -1.0, 2.0, -2.0, 2.5, -3.0, 7.0):
        assert orc.kernel(BICUBIC, t) == 0.0


@pytest.mark.parametrize("f", list(np.linspace(0.0, 1.0, 49)))
def test_keys_partition_and_polynomial_reproduction(orc, f):
    # Keys' cubic with a = -1/2 reproduces polynomials up to degree 2; any other a fails degree 2,
    # and a wrong constant term on 1<|t|<2 fails degree 0.
    ts = range(-3, 5)
    w = [orc.kernel(BICUBIC, f - t) for t in ts]
    assert abs(sum(w) - 1.0) < 1e-14
    assert abs(sum(t * wi for t, wi in zip(ts, w)) - f) < 1e-14
    assert abs(sum(t * t * wi for t, wi in zip(ts, w)) - f * f) < 1e-13


def test_keys_kernel_is_c1(orc):
    h = 1e-7
    for knot in (1.0, 2.0):
        left = orc.kernel(BICUBIC, knot - h)
        right = orc.kernel(BICUBIC, knot + h)
        assert abs(left - right) < 1e-6  # continuous
        dl = (orc.kernel(BICUBIC, knot - h) - orc.kernel(BICUBIC, knot - 2 * h)) / h
        dr = (orc.kernel(BICUBIC, knot + 2 * h) - orc.kernel(BICUBIC, knot + h)) / h
        assert abs(dl - dr) < 1e-5  # continuous first derivative
    # symmetric
    for t in np.linspace(0, 2.5, 11):
        assert orc.kernel(BICUBIC, t) == orc.kernel(BICUBIC, -t)


@pytest.mark.parametrize("f", list(np.linspace(0.0, 1.0, 17)))
def test_bilinear_kernel_hat(orc, f):
    assert orc.kernel(BILINEAR, 0.0) == 1.0 and orc.kernel(BILINEAR, 1.0) == 0.0
    ts = range(-2, 4)
    w = [orc.kernel(BILINEAR, f - t) for t in ts]
    assert abs(sum(w) - 1.0) < 1e-15
    assert abs(sum(t * wi for t, wi in zip(ts, w)) - f) < 1e-15
    assert all(wi >= 0 for wi in w)


# ------------------------------------------------- geometry and weight tables

def test_output_lengths_of_the_workloads(orc):
    assert orc.out_len(64, 3, 2) == 96
    assert orc.out_len(1080, 2, 3) == 720 and orc.out_len(1920, 2, 3) == 1280
    assert orc.out_len(1080, 4, 3) == 1440 and orc.out_len(1920, 4, 3) == 2560
    assert orc.out_len(1080, 3, 2) == 1620 and orc.out_len(1920, 3, 2) == 2880
    assert orc.out_len(256, 5, 4) == 320 and orc.out_len(256, 3, 2) == 384
    assert orc.out_len(8192, 7, 5) == 11468
    assert orc.out_len(17, 5, 4) == 21 and orc.out_len(23, 5, 4) == 28
    assert orc.out_len(0, 3, 2) == 0 and orc.out_len(1, 1, 2) == 0


@pytest.mark.parametrize("method,r,s,K,L", [(BILINEAR, 3, 2, 1, 0), (BICUBIC, 3, 2, 2, 1), (BICUBIC, 2, 3, 3, 2),
                                              (BICUBIC, 4, 3, 3, 2), (BILINEAR, 5, 4, 2, 0), (BICUBIC, 7, 5, 4, 2)])
def test_kmin_and_left_offset(orc, method, r, s, K, L):
    assert orc.kmin(method, s) == K
    assert orc.left_offset(K, s) == L


@pytest.mark.parametrize("r,s", RATIOS)
@pytest.mark.parametrize("method", (BILINEAR, BICUBIC))
def test_weight_table_moments(orc, method, r, s):
    # every phase j interpolates at j s / r: unit mass, first moment j s / r (second for Keys)
    for extra in (0, 1):
        K = orc.kmin(method, s) + extra
        W, _ = orc.make_weights(method, r, s, K)
        L = orc.left_offset(K, s)
        pos = np.arange(W.shape[1]) - L
        for j in range(r):
            f = j * s / r
            assert abs(W[j].sum() - 1.0) < 1e-14
            assert abs((W[j] * pos).sum() - f) < 1e-13
            if method == BICUBIC:
                assert abs((W[j] * pos * pos).sum() - f * f) < 1e-12


@pytest.mark.parametrize("r,s", RATIOS)
def test_nearest_table_rounds_half_up(orc, r, s):
    W, K = orc.make_weights(NEAREST, r, s)
    L = orc.left_offset(K, s)
    for j in range(r):
        (m,) = np.nonzero(W[j])[0]
        target = Fraction(j * s, r) + Fraction(1, 2)
        assert m - L == math.floor(target)
        assert W[j, m] == 1.0


def test_k_below_minimum_is_rejected(orc):
    with pytest.raises(ValueError):
        orc.make_weights(BICUBIC, 4, 3, 2)


# ------------------------------------------------- printed examples (P1, P2)

def _phase_blocks(orc, method, r, s):
    """All r*r 2D phase kernels (outer products), each cut to the 2x2 block at its
    floor taps, together with the kernel's total mass outside that block."""
    W, K = orc.make_weights(method, r, s)
    L = orc.left_offset(K, s)
    out = []
    for jy in range(r):
        for jx in range(r):
            k2 = np.outer(W[jy], W[jx])
            by, bx = (jy * s) // r + L, (jx * s) // r + L
            block = k2[by:by + 2, bx:bx + 2]
            out.append((block, np.abs(k2).sum() - np.abs(block).sum()))
    return out


@pytest.mark.parametrize("method,name", [(NEAREST, "nearest"), (BILINEAR, "bilinear")])
def test_printed_sec5_kernels_appear(orc, method, name):
    gold = json.load(open(GOLDEN))
    blocks = _phase_blocks(orc, method, gold["r"], gold["s"])
    for key in ("W11", "W13"):
        printed = np.array(gold[name][key])
        hits = [b for b, rest in blocks if np.array_equal(np.round(b, 2), printed) and rest < 1e-15]
        assert hits, f"{name} {key} {printed.tolist()} not among the 3/2 phase kernels"


def test_printed_bicubic_matrices_are_not_keys(orc):
    # recorded reading: the printed 3x3 bicubic matrices are not Keys weights (no phase gives them)
    gold = json.load(open(GOLDEN))["bicubic_printed_not_reproducible"]
    W, K = orc.make_weights(BICUBIC, 3, 2)
    for key in ("W11", "W13"):
        printed = np.array(gold[key])
        for jy in range(3):
            for jx in range(3):
                k2 = np.outer(W[jy], W[jx])
                for oy in range(k2.shape[0] - 2):
                    for ox in range(k2.shape[1] - 2):
                        assert not np.array_equal(np.round(k2[oy:oy + 3, ox:ox + 3], 2), printed)


# ------------------------------------------- exact-rational brute force (P7)

def _ext(q, n, pad):
    """Sec. 3 padding rules restated: replicate, constant (None), reflect about the edge samples."""
    if 0 <= q < n:
        return q
    if pad == CONST:
        return None
    if pad == REPL:
        return 0 if q < 0 else n - 1
    if n == 1:
        return 0
    while not 0 <= q < n:
        q = -q if q < 0 else 2 * (n - 1) - q
    return q


def _sample(at, p, method):
    """Value at position p (a Fraction) from the neighbours given by at(q)."""
    b = math.floor(p)
    f = p - b
    if method == NEAREST:
        return at(math.floor(p + Fraction(1, 2)))
    if method == BILINEAR:
        return at(b) + f * (at(b + 1) - at(b))
    # Catmull-Rom spline through four neighbours (the cubic convolution of Keys with a = -1/2)
    p0, p1, p2, p3 = at(b - 1), at(b), at(b + 1), at(b + 2)
    return (2 * p1 + (p2 - p0) * f + (2 * p0 - 5 * p1 + 4 * p2 - p3) * f * f
            + (3 * p1 - p0 - 3 * p2 + p3) * f * f * f) / 2


def _brute_1d(x, r, s, method, pad, c):
    xs = [Fraction(float(v)) for v in x]
    cf = Fraction(float(c))

    def at(q):
        k = _ext(q, len(xs), pad)
        return cf if k is None else xs[k]

    return [_sample(at, Fraction(o * s, r), method) for o in range(len(xs) * r // s)]


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
def test_bruteforce_1d_all_ratios(orc, method, pad):
    rng = np.random.default_rng(100 + 3 * method + pad)
    for n in range(1, 10):
        for r, s in RATIOS:
            x = rng.random(n)
            c = 0.37
            want = np.array([float(v) for v in _brute_1d(x, r, s, method, pad, c)])
            got = orc.resize(x[None, None], [dict(r=r, s=s, method=method)], pad=pad, pad_value=c)[0, 0]
            assert got.shape == want.shape
            if method == NEAREST:
                assert np.array_equal(got, want)
            else:
                assert np.max(np.abs(got - want), initial=0.0) <= 1e-15 * 2, (n, r, s)


def _brute_nd(x, ratios, method, pad, c):
    """Tensor-product sampling, one axis after the other; out-of-range rows of the
    constant pad are rows of c (the ND extension of Sec. 4)."""
    nd = x.ndim
    cur = np.vectorize(lambda v: Fraction(float(v)), otypes=[object])(x)
    cf = Fraction(float(c))
    for ax in range(nd - 1, -1, -1):
        r, s = ratios[ax]
        n = cur.shape[ax]
        no = n * r // s
        moved = np.moveaxis(cur, ax, -1)
        out = np.empty(moved.shape[:-1] + (no,), dtype=object)
        for idx in np.ndindex(moved.shape[:-1]):
            line = moved[idx]

            def at(q, line=line):
                k = _ext(q, n, pad)
                return cf if k is None else line[k]

            for o in range(no):
                out[idx + (o,)] = _sample(at, Fraction(o * s, r), method)
        cur = np.moveaxis(out, -1, ax)
    return np.vectorize(float, otypes=[np.float64])(cur)


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
def test_bruteforce_2d_3d(orc, method, pad):
    rng = np.random.default_rng(7 + method + 10 * pad)
    cases = [((5, 7), [(3, 2), (2, 3)]), ((4, 6), [(5, 4), (7, 5)]), ((3, 2), [(2, 1), (1, 2)]),
             ((3, 4, 5), [(3, 2), (2, 3), (4, 3)]), ((2, 3, 3), [(5, 2), (1, 1), (2, 11)])]
    for shape, ratios in cases:
        x = rng.random(shape)
        want = _brute_nd(x, ratios, method, pad, -0.25)
        got = orc.resize(x[None, None], [dict(r=r, s=s, method=method) for r, s in ratios],
                         pad=pad, pad_value=-0.25)[0, 0]
        assert got.shape == want.shape
        if method == NEAREST:
            assert np.array_equal(got, want)
        else:
            assert np.max(np.abs(got - want), initial=0) <= 4e-15


# ------------------------------------- the paper's construction (P4), torch FP64

def _construction(x, axes, pad, c):
    """Sec. 3.1 / Sec. 4 pseudocode with library ops: pad, N-d conv with prod(r) output
    channels per input channel and stride s, N-d pixelshuffle (last axis fastest), crop."""
    import torch
    import torch.nn.functional as F

    x = torch.from_numpy(x)
    n, C = x.shape[:2]
    sp = list(x.shape[2:])
    nd = len(sp)
    pads, crops, Ts, rs, ss = [], [], [], [], []
    Ws = []
    for a, ax in enumerate(axes):
        r, s, K = ax["r"], ax["s"], ax["K"]
        T, L = 2 * K + 1, K - s // 2
        no = sp[a] * r // s
        nw = -(-no // r)
        right = max(0, (nw - 1) * s + T - L - sp[a])
        pads.append((L, right))
        crops.append((no, nw))
        Ts.append(T)
        rs.append(r)
        ss.append(s)
        w = torch.from_numpy(np.asarray(ax["w"], dtype=np.float64))
        Ws.append(w if w.dim() == 3 else w.unsqueeze(0).expand(C, r, T))
    flat = []
    for L, R in reversed(pads):
        flat += [L, R]
    mode = {REPL: "replicate", CONST: "constant", REFL: "reflect"}[pad]
    if mode == "constant":
        xp = F.pad(x, flat, mode="constant", value=c)
    else:
        xp = F.pad(x, flat, mode=mode)
    P = int(np.prod(rs))
    weight = torch.empty((C * P, 1) + tuple(Ts), dtype=torch.float64)
    for ch in range(C):
        for ph in range(P):
            js, rem = [], ph
            for r in reversed(rs):
                js.append(rem % r)
                rem //= r
            js = js[::-1]
            k = Ws[0][ch, js[0]]
            for a in range(1, nd):
                k = torch.tensordot(k, Ws[a][ch, js[a]], dims=0)
            weight[ch * P + ph, 0] = k
    conv = {1: F.conv1d, 2: F.conv2d, 3: F.conv3d}[nd]
    h = conv(xp, weight, stride=tuple(ss), groups=C)  # hidden layer: [n, C*P, windows...]
    nws = [cw[1] for cw in crops]
    h = h[(slice(None), slice(None)) + tuple(slice(0, w) for w in nws)]
    h = h.reshape([n, C] + rs + nws)
    perm = [0, 1]
    for a in range(nd):
        perm += [2 + nd + a, 2 + a]
    y = h.permute(perm).reshape([n, C] + [w * r for w, r in zip(nws, rs)])
    y = y[(slice(None), slice(None)) + tuple(slice(0, cw[0]) for cw in crops)]
    return y.numpy()


CONSTRUCTION_CASES = [
    ((9,), [(3, 2)]), ((11,), [(2, 3)]), ((7,), [(1, 2)]), ((13,), [(27, 11)]),
    ((9, 10), [(3, 2), (3, 2)]), ((12, 13), [(2, 3), (4, 3)]), ((8, 9), [(5, 4), (7, 5)]),
    ((6, 5), [(2, 1), (3, 1)]), ((5, 6, 7), [(3, 2), (3, 2), (3, 2)]), ((4, 5, 6), [(2, 3), (5, 4), (1, 1)]),
]


@pytest.mark.parametrize("spatial,ratios", CONSTRUCTION_CASES)
@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("pad", (REPL, CONST))
def test_direct_formula_equals_construction(orc, spatial, ratios, method, pad):
    rng = np.random.default_rng(len(spatial) * 1000 + method * 10 + pad)
    x = rng.random((2, 3) + spatial)
    axes = []
    for r, s in ratios:
        W, K = orc.make_weights(method, r, s, orc.kmin(method, s) + 1)  # K above the minimum on purpose
        axes.append(dict(r=r, s=s, method=method, K=K, w=W))
    want = _construction(x, axes, pad, 0.3)
    direct = orc.resize(x, [dict(r=r, s=s, method=method) for r, s in ratios], pad=pad, pad_value=0.3)
    assert direct.shape == want.shape
    assert np.max(np.abs(direct - want), initial=0) <= 1e-13
    if method == NEAREST:
        assert np.array_equal(direct, want)


@pytest.mark.parametrize("spatial,ratios", CONSTRUCTION_CASES)
@pytest.mark.parametrize("pad", (REPL, CONST))
def test_polyphase_learnable_equals_construction(orc, spatial, ratios, pad):
    rng = np.random.default_rng(5 + len(spatial) + pad)
    C = 3
    x = rng.standard_normal((2, C) + spatial)
    axes = []
    for a, (r, s) in enumerate(ratios):
        K = orc.kmin(BILINEAR, s) + (a % 2)
        per_channel = a % 2 == 0
        w = rng.standard_normal((C, r, 2 * K + 1) if per_channel else (r, 2 * K + 1))
        axes.append(dict(r=r, s=s, method=BILINEAR, K=K, w=w))
    want = _construction(x, axes, pad, -0.7)
    got = orc.resize(x, axes, pad=pad, pad_value=-0.7, polyphase=True)
    scale = np.abs(x).max() * np.prod([np.abs(a["w"]).sum(-1).max() for a in axes])
    assert np.max(np.abs(got - want)) <= 1e-13 * scale


@pytest.mark.parametrize("spatial,ratios", CONSTRUCTION_CASES)
@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
def test_direct_equals_polyphase_at_table_weights(orc, spatial, ratios, method, pad):
    rng = np.random.default_rng(11)
    x = rng.random((1, 2) + spatial)
    axes = [dict(r=r, s=s, method=method) for r, s in ratios]
    a = orc.resize(x, axes, pad=pad, pad_value=0.5)
    b = orc.resize(x, axes, pad=pad, pad_value=0.5, polyphase=True)
    assert np.max(np.abs(a - b), initial=0) <= 1e-15 * 4
    if method == NEAREST:
        assert np.array_equal(a, b)


# ------------------------------------------------- scipy linear interpolation

@pytest.mark.parametrize("pad,mode", [(REPL, "nearest"), (REFL, "mirror"), (CONST, "grid-constant")])
def test_bilinear_matches_scipy_map_coordinates(orc, pad, mode):
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(3)
    for shape, ratios in [((11, 13), [(3, 2), (2, 3)]), ((9, 8), [(4, 3), (7, 5)]), ((6, 7, 5), [(3, 2), (5, 4), (2, 3)])]:
        x = rng.random(shape)
        outs = [n * r // s for n, (r, s) in zip(shape, ratios)]
        grids = np.meshgrid(*[np.arange(o) * s / r for o, (r, s) in zip(outs, ratios)], indexing="ij")
        want = ndimage.map_coordinates(x, grids, order=1, mode=mode, cval=0.2)
        got = orc.resize(x[None, None], [dict(r=r, s=s, method=BILINEAR) for r, s in ratios],
                         pad=pad, pad_value=0.2)[0, 0]
        assert np.max(np.abs(got - want)) < 1e-12


# ------------------------------------------------------------ invariants (P6)

@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("r,s", RATIOS)
def test_constant_image_preserved(orc, method, r, s):
    x = np.full((1, 1, 7, 9), 0.625)
    for pad, c in ((REPL, 0.0), (REFL, 0.0), (CONST, 0.625)):
        y = orc.resize(x, [dict(r=r, s=s, method=method)] * 2, pad=pad, pad_value=c)
        assert np.max(np.abs(y - 0.625), initial=0) <= 4e-15  # rounding of 16 terms


@pytest.mark.parametrize("method", (BILINEAR, BICUBIC))
@pytest.mark.parametrize("r,s", RATIOS)
def test_ramp_preserved_inside(orc, method, r, s):
    n = 23
    x = 0.75 * np.arange(n) - 2.0
    y = orc.resize(x[None, None], [dict(r=r, s=s, method=method)])[0, 0]
    R = 2 if method == BICUBIC else 1
    for o in range(len(y)):
        b = (o * s) // r
        if b - R + 1 >= 0 and b + R <= n - 1:
            assert abs(y[o] - (0.75 * o * s / r - 2.0)) < 1e-13
    if method == BICUBIC:
        q = (np.arange(n) - 4.0) ** 2
        yq = orc.resize(q[None, None], [dict(r=r, s=s, method=method)])[0, 0]
        for o in range(len(yq)):
            b = (o * s) // r
            if b - 1 >= 0 and b + 2 <= n - 1:
                assert abs(yq[o] - (o * s / r - 4.0) ** 2) < 1e-12


@pytest.mark.parametrize("method", METHODS)
def test_r_equals_s_is_identity(orc, method):
    x = np.random.default_rng(0).standard_normal((2, 2, 6, 7))
    for k in (1, 2, 3, 5):
        for pad in (REPL, CONST, REFL):
            y = orc.resize(x, [dict(r=k, s=k, method=method)] * 2, pad=pad, pad_value=9.0)
            assert np.array_equal(y, x)


@pytest.mark.parametrize("method", METHODS)
def test_unreduced_ratio_is_the_same_operator(orc, method):
    x = np.random.default_rng(1).random((1, 2, 9, 11))
    for r, s in ((3, 2), (2, 3), (5, 4)):
        a = orc.resize(x, [dict(r=r, s=s, method=method)] * 2)
        b = orc.resize(x, [dict(r=2 * r, s=2 * s, method=method)] * 2)
        c = orc.resize(x, [dict(r=3 * r, s=3 * s, method=method)] * 2)
        assert np.array_equal(a, b) and np.array_equal(a, c)


@pytest.mark.parametrize("r,s", RATIOS)
def test_nearest_outputs_are_input_samples(orc, r, s):
    x = np.random.default_rng(2).random((1, 1, 8, 9))
    y = orc.resize(x, [dict(r=r, s=s, method=NEAREST)] * 2)
    assert np.isin(y, x).all()


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
def test_separable_rows_then_columns(orc, method, pad):
    x = np.random.default_rng(4).random((1, 1, 10, 12))
    ay, ax = dict(r=4, s=3, method=method), dict(r=2, s=3, method=method)
    full = orc.resize(x, [ay, ax], pad=pad, pad_value=0.1)[0, 0]
    rows = orc.resize(x[0, 0][:, None, :], [ax], pad=pad, pad_value=0.1)[:, 0, :]    # [H, Wo]
    cols = orc.resize(rows.T[:, None, :], [ay], pad=pad, pad_value=0.1)[:, 0, :].T   # [Ho, Wo]
    assert np.max(np.abs(full - cols)) <= 1e-15 * 4


@pytest.mark.parametrize("r", (2, 3, 4))
def test_s1_is_subpixel_upsampling(orc, r):
    # A14: FCFS(r/1) = pixelshuffle(conv(x~, W, stride 1)) with the same phase kernels
    x = np.random.default_rng(r).random((1, 2, 6, 5))
    for method in METHODS:
        W, K = orc.make_weights(method, r, 1)
        axes = [dict(r=r, s=1, method=method, K=K, w=W)] * 2
        want = _construction(x, axes, REPL, 0.0)
        got = orc.resize(x, [dict(r=r, s=1, method=method)] * 2)
        assert np.max(np.abs(got - want)) <= 1e-14


def test_empty_and_degenerate_shapes(orc):
    x = np.random.default_rng(0).random((1, 1, 1, 1))
    assert orc.resize(x, [dict(r=1, s=2, method=BILINEAR)] * 2).shape == (1, 1, 0, 0)
    y = orc.resize(x, [dict(r=3, s=1, method=BICUBIC)] * 2)
    assert y.shape == (1, 1, 3, 3) and np.allclose(y, x[0, 0, 0, 0], rtol=0, atol=4e-15)
    assert orc.resize(np.zeros((0, 3, 4, 4)), [dict(r=3, s=2)] * 2).shape == (0, 3, 6, 6)


# -------------------------------------------------------------- adjoint (P8)

def _learnable_axes(rng, C, ratios):
    axes = []
    for a, (r, s) in enumerate(ratios):
        K = max(1, (s + 1) // 2) + a % 2
        w = rng.standard_normal((C, r, 2 * K + 1) if a % 2 == 0 else (r, 2 * K + 1))
        axes.append(dict(r=r, s=s, K=K, w=w))
    return axes


@pytest.mark.parametrize("spatial,ratios", [((13,), [(3, 2)]), ((9, 11), [(5, 4), (2, 3)]),
                                            ((6, 7, 5), [(3, 2), (4, 3), (1, 2)])])
@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
def test_adjoint_dot_product(orc, spatial, ratios, pad):
    rng = np.random.default_rng(17)
    C = 2
    axes = _learnable_axes(rng, C, ratios)
    x = rng.standard_normal((2, C) + spatial)
    y = orc.resize(x, axes, pad=pad, pad_value=0.0, polyphase=True)
    g = rng.standard_normal(y.shape)
    dx = orc.adjoint_dx(g, spatial, axes, pad=pad)
    lhs, rhs = np.vdot(y, g), np.vdot(x, dx)
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.abs(y).sum())


@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
def test_adjoint_gather_equals_scatter(orc, pad):
    rng = np.random.default_rng(23)
    spatial, ratios = (7, 9), [(5, 4), (2, 3)]
    axes = _learnable_axes(rng, 2, ratios)
    g = rng.standard_normal((1, 2) + tuple(n * r // s for n, (r, s) in zip(spatial, ratios)))
    full = orc.adjoint_dx(g, spatial, axes, pad=pad)
    at = orc.adjoint_dx_at(g, spatial, axes, np.arange(full.size), pad=pad)
    assert np.max(np.abs(at - full.ravel())) <= 1e-13


@pytest.mark.parametrize("spatial,ratios", [((29,), [(7, 5)]), ((9, 11), [(5, 4), (2, 3)]),
                                            ((6, 7, 5), [(3, 2), (4, 3), (1, 2)])])
@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
def test_resize_at_decodes_flat_indices(orc, spatial, ratios, pad):
    # the sampled full-size GPU parity rests on resize_at; it must return exactly the
    # entries of the full result at the flat indices of [n][c][out...] (plane, channel of
    # the per-channel weights, each spatial output index), for every evaluation form
    rng = np.random.default_rng(29)
    n, C = 3, 4
    x = rng.standard_normal((n, C) + spatial)
    forms = [(_learnable_axes(rng, C, ratios), True)]
    for m in METHODS:
        for align in (0, 1, 2):
            forms.append(([dict(r=r, s=s, method=m, align=align) for r, s in ratios], False))
    forms.append(([dict(r=r, s=s, method=BICUBIC, cubic_a=-0.75) for r, s in ratios], False))
    forms.append(([dict(r=r, s=s, method=BILINEAR) for r, s in ratios], True))
    for axes, poly in forms:
        full = orc.resize(x, axes, pad=pad, pad_value=0.25, polyphase=poly)
        idx = np.concatenate([rng.integers(0, full.size, 300), [0, full.size - 1]])
        at = orc.resize_at(x, axes, idx, pad=pad, pad_value=0.25, polyphase=poly)
        assert np.array_equal(at, full.ravel()[idx])
        # the decode is not a no-op: outputs of other planes / channels differ
        assert not np.array_equal(at, full.ravel()[(idx + full[0, 0].size) % full.size])


def _fd_slice(orc):
    # 1x2x17x23 slice, scale 5/4 on both axes, per-channel taps initialised to bilinear and perturbed
    rng = np.random.default_rng(31)
    W, K = orc.make_weights(BILINEAR, 5, 4)
    axes = [dict(r=5, s=4, K=K, w=np.stack([W, W]) + 0.05 * rng.standard_normal((2, 5, 2 * K + 1)))
            for _ in range(2)]
    x = rng.standard_normal((1, 2, 17, 23))
    g = rng.standard_normal((1, 2, 21, 28))
    return axes, x, g


def test_finite_difference_dx(orc):
    axes, x, g = _fd_slice(orc)
    dx = orc.adjoint_dx(g, x.shape[2:], axes)
    rng = np.random.default_rng(0)
    h = 1e-6
    picks = [tuple(rng.integers(0, d) for d in x.shape) for _ in range(40)] + [(0, 0, 0, 0), (0, 1, 16, 22)]
    for p in picks:
        xp, xm = x.copy(), x.copy()
        xp[p] += h
        xm[p] -= h
        fd = (np.vdot(orc.resize(xp, axes, polyphase=True), g) - np.vdot(orc.resize(xm, axes, polyphase=True), g)) / (2 * h)
        assert abs(fd - dx[p]) <= 1e-6 * max(1.0, abs(dx[p]))


@pytest.mark.parametrize("pad", (REPL, CONST))
def test_finite_difference_dw(orc, pad):
    axes, x, g = _fd_slice(orc)
    dws = orc.weight_grad(x, g, axes, pad=pad, pad_value=0.4)
    rng = np.random.default_rng(1)
    h = 1e-6
    for a in range(2):
        for _ in range(12):
            p = tuple(rng.integers(0, d) for d in axes[a]["w"].shape)
            loss = []
            for sign in (1, -1):
                ax2 = [dict(v) for v in axes]
                w = ax2[a]["w"].copy()
                w[p] += sign * h
                ax2[a]["w"] = w
                loss.append(np.vdot(orc.resize(x, ax2, pad=pad, pad_value=0.4, polyphase=True), g))
            fd = (loss[0] - loss[1]) / (2 * h)
            assert abs(fd - dws[a][p]) <= 1e-6 * max(1.0, abs(fd))


def test_shared_weight_gradient_sums_channels(orc):
    rng = np.random.default_rng(5)
    W, K = orc.make_weights(BILINEAR, 3, 2)
    x = rng.standard_normal((2, 3, 6, 7))
    g = rng.standard_normal((2, 3, 9, 10))
    shared = [dict(r=3, s=2, K=K, w=W)] * 2
    per = [dict(r=3, s=2, K=K, w=np.stack([W] * 3))] * 2
    ds = orc.weight_grad(x, g, shared)
    dp = orc.weight_grad(x, g, per)
    for a in range(2):
        assert np.allclose(ds[a], dp[a].sum(0), rtol=0, atol=1e-12)


# ------------------------------------------- sample-alignment variants (P5)
# Not the paper's sampling: the half-pixel-centre and floor-nearest conventions of
# common resize libraries.  Pinned to PyTorch's CPU interpolation in float64, which
# uses the same positions when given scale_factor (not size).

HALF, FLOOR = 1, 2
VAR_RATIOS = [(3, 2), (2, 3), (4, 3), (5, 4), (7, 5), (5, 2), (1, 2), (2, 1), (2, 11)]


def _torch_interp(x, ratio, mode, ndim):
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    sf = (ratio[0] / ratio[1],) * ndim
    kw = {} if mode in ("nearest", "nearest-exact") else {"align_corners": False}
    return F.interpolate(torch.from_numpy(x), scale_factor=sf, mode=mode, recompute_scale_factor=False, **kw).numpy()


@pytest.mark.parametrize("ratio", VAR_RATIOS)
def test_half_pixel_bilinear_matches_library_interpolation(orc, ratio):
    x = np.random.default_rng(41).random((1, 2, 13, 17))
    want = _torch_interp(x, ratio, "bilinear", 2)
    got = orc.resize(x, [dict(r=ratio[0], s=ratio[1], method=BILINEAR, align=HALF)] * 2, pad=REPL)
    assert got.shape == want.shape
    assert np.abs(got - want).max() <= 1e-12


@pytest.mark.parametrize("ratio", VAR_RATIOS)
def test_half_pixel_bicubic_a075_matches_library_interpolation(orc, ratio):
    # the library's cubic has Keys a = -3/4 and clamps indices at the border (replicate)
    x = np.random.default_rng(42).random((1, 2, 13, 17))
    want = _torch_interp(x, ratio, "bicubic", 2)
    got = orc.resize(x, [dict(r=ratio[0], s=ratio[1], method=BICUBIC, align=HALF, cubic_a=-0.75)] * 2, pad=REPL)
    assert got.shape == want.shape
    assert np.abs(got - want).max() <= 1e-12


@pytest.mark.parametrize("ratio", VAR_RATIOS)
@pytest.mark.parametrize("align,mode", [(FLOOR, "nearest"), (HALF, "nearest-exact")])
def test_nearest_variants_match_library_interpolation(orc, ratio, align, mode):
    x = np.random.default_rng(43).random((2, 1, 11, 19))
    want = _torch_interp(x, ratio, mode, 2)
    got = orc.resize(x, [dict(r=ratio[0], s=ratio[1], method=NEAREST, align=align)] * 2, pad=REPL)
    assert got.shape == want.shape
    assert np.array_equal(got, want)


@pytest.mark.parametrize("ratio", [(3, 2), (2, 3), (5, 4)])
def test_half_pixel_linear_1d_matches_library_interpolation(orc, ratio):
    x = np.random.default_rng(44).random((1, 3, 29))
    want = _torch_interp(x, ratio, "linear", 1)
    got = orc.resize(x, [dict(r=ratio[0], s=ratio[1], method=BILINEAR, align=HALF)], pad=REPL)
    assert np.abs(got - want).max() <= 1e-12


def test_floor_nearest_s1_is_repeat_interleave(orc):
    # floor-nearest at r/1 repeats every sample r times (the paper's rounding does not)
    x = np.random.default_rng(45).random((1, 1, 9))
    for r in (2, 3, 4):
        got = orc.resize(x, [dict(r=r, s=1, method=NEAREST, align=FLOOR)])
        assert np.array_equal(got[0, 0], np.repeat(x[0, 0], r))


@pytest.mark.parametrize("method", (BILINEAR, BICUBIC))
def test_variant_invariants(orc, method):
    rng = np.random.default_rng(46)
    x = rng.random((1, 1, 12, 10))
    # r = s: the half-pixel position is the sample itself
    same = orc.resize(x, [dict(r=3, s=3, method=method, align=HALF)] * 2)
    assert np.abs(same - x).max() <= 1e-15
    # floor alignment only changes nearest
    a = orc.resize(x, [dict(r=4, s=3, method=method, align=FLOOR)] * 2)
    b = orc.resize(x, [dict(r=4, s=3, method=method)] * 2)
    assert np.array_equal(a, b)
    # constants are preserved, any Keys parameter
    c = np.full((1, 1, 8, 8), 0.37)
    for ka in (-0.5, -0.75):
        y = orc.resize(c, [dict(r=5, s=4, method=method, align=HALF, cubic_a=ka)] * 2, pad=REFL)
        assert np.abs(y - 0.37).max() <= 1e-14
    # the polyphase evaluation refuses fixed-method variants (its tables are the paper's)
    with pytest.raises(ValueError):
        orc.resize(x, [dict(r=4, s=3, method=method, align=HALF)] * 2, polyphase=True)


@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
@pytest.mark.parametrize("axes", [[dict(r=3, s=2, method=BICUBIC, align=HALF, cubic_a=-0.75)] * 2,
                                  [dict(r=2, s=3, method=BILINEAR, align=HALF), dict(r=5, s=4, method=NEAREST, align=FLOOR)],
                                  [dict(r=4, s=3, method=NEAREST, align=HALF)] * 2])
def test_variant_adjoint_dot_product(orc, pad, axes):
    rng = np.random.default_rng(47)
    x = rng.standard_normal((2, 2, 9, 11))
    y = orc.resize(x, axes, pad=pad, pad_value=0.0)
    g = rng.standard_normal(y.shape)
    dx = orc.adjoint_dx(g, (9, 11), axes, pad=pad)
    lhs, rhs = np.vdot(y, g), np.vdot(x, dx)
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.abs(y).sum())


# -------------------------------------------- non-separable 2D kernels (f2)
# One learnable T_y x T_x kernel per phase pair (Sec. 4's ND convolution without
# the outer-product restriction).  Pinned to the paper's construction built from
# PyTorch CPU library ops in float64 (pad -> grouped strided conv2d -> pixel
# shuffle -> crop), whose autograd also pins the input and weight gradients.

def _full2d_construction(x, w, ratios, Ks, pad, pad_value):
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    n, c, H, W = x.shape
    (ry, sy), (rx, sx) = ratios
    Ty, Tx = 2 * Ks[0] + 1, 2 * Ks[1] + 1
    Ly, Lx = Ks[0] - sy // 2, Ks[1] - sx // 2
    Ho, Wo = H * ry // sy, W * rx // sx
    nwy, nwx = -(-Ho // ry), -(-Wo // rx)
    ry_pad = max(0, (nwy - 1) * sy - Ly + Ty - H)
    rx_pad = max(0, (nwx - 1) * sx - Lx + Tx - W)
    xt = x if isinstance(x, torch.Tensor) else torch.from_numpy(x)
    mode = {REPL: "replicate", CONST: "constant", REFL: "reflect"}[pad]
    kw = {"value": pad_value} if pad == CONST else {}
    # left pads may be negative (a window that starts inside the image): crop instead
    xp = F.pad(xt, (max(Lx, 0), rx_pad, max(Ly, 0), ry_pad), mode=mode, **kw)
    xp = xp[:, :, max(-Ly, 0):, max(-Lx, 0):]
    wt = w if isinstance(w, torch.Tensor) else torch.from_numpy(w)
    if wt.dim() == 4:
        wt = wt.unsqueeze(0).expand(c, *wt.shape)
    k = wt.reshape(c * ry * rx, 1, Ty, Tx)
    z = F.conv2d(xp, k, stride=(sy, sx), groups=c)[:, :, :nwy, :nwx]
    z = z.reshape(n, c, ry, rx, nwy, nwx).permute(0, 1, 4, 2, 5, 3).reshape(n, c, nwy * ry, nwx * rx)
    return z[:, :, :Ho, :Wo]


FULL_CASES = [(((3, 2), (2, 3)), (1, 2)), (((5, 4), (5, 4)), (2, 2)), (((2, 1), (3, 2)), (1, 1)), (((4, 3), (1, 2)), (2, 1))]


@pytest.mark.parametrize("ratios,Ks", FULL_CASES)
@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
@pytest.mark.parametrize("per_channel", (True, False))
def test_full2d_matches_construction(orc, ratios, Ks, pad, per_channel):
    rng = np.random.default_rng(51)
    C = 3
    (ry, _), (rx, _) = ratios
    shape = (ry, rx, 2 * Ks[0] + 1, 2 * Ks[1] + 1)
    w = rng.standard_normal(((C,) + shape) if per_channel else shape)
    x = rng.standard_normal((2, C, 11, 13))
    axes = [dict(r=r, s=s, K=K) for (r, s), K in zip(ratios, Ks)]
    got = orc.resize_full2d(x, axes, w, pad=pad, pad_value=0.4)
    want = _full2d_construction(x, w, ratios, Ks, pad, 0.4).numpy()
    assert got.shape == want.shape
    assert np.abs(got - want).max() <= 1e-12 * (1 + np.abs(want).max())


@pytest.mark.parametrize("ratios,Ks", FULL_CASES[:2])
@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
def test_full2d_gradients_match_construction_autograd(orc, ratios, Ks, pad):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(52)
    C = 2
    (ry, _), (rx, _) = ratios
    w = torch.tensor(rng.standard_normal((C, ry, rx, 2 * Ks[0] + 1, 2 * Ks[1] + 1)), requires_grad=True)
    x = torch.tensor(rng.standard_normal((2, C, 10, 12)), requires_grad=True)
    y = _full2d_construction(x, w, ratios, Ks, pad, 0.0)
    g = torch.tensor(rng.standard_normal(tuple(y.shape)))
    (y * g).sum().backward()
    axes = [dict(r=r, s=s, K=K) for (r, s), K in zip(ratios, Ks)]
    dx = orc.adjoint_full2d(g.numpy(), (10, 12), axes, w.detach().numpy(), pad=pad)
    dw = orc.weight_grad_full2d(x.detach().numpy(), g.numpy(), axes, True, pad=pad)
    assert np.abs(dx - x.grad.numpy()).max() <= 1e-12 * (1 + np.abs(dx).max())
    assert np.abs(dw - w.grad.numpy()).max() <= 1e-12 * (1 + np.abs(dw).max())


def test_full2d_outer_product_is_the_separable_layer(orc):
    rng = np.random.default_rng(53)
    C = 2
    wy = rng.standard_normal((C, 3, 5))
    wx = rng.standard_normal((C, 2, 3))
    w = np.einsum("cjm,ckn->cjkmn", wy, wx)
    x = rng.standard_normal((1, C, 12, 14))
    sep = orc.resize(x, [dict(r=3, s=2, K=2, w=wy), dict(r=2, s=3, K=1, w=wx)], pad=REFL, polyphase=True)
    full = orc.resize_full2d(x, [dict(r=3, s=2, K=2), dict(r=2, s=3, K=1)], w, pad=REFL)
    assert np.abs(sep - full).max() <= 1e-13 * (1 + np.abs(sep).max())
    # shared kernels sum the channels' weight gradients
    g = rng.standard_normal(full.shape)
    axes = [dict(r=3, s=2, K=2), dict(r=2, s=3, K=1)]
    per = orc.weight_grad_full2d(x, g, axes, True, pad=REFL)
    shared = orc.weight_grad_full2d(x, g, axes, False, pad=REFL)
    assert np.abs(per.sum(0) - shared).max() <= 1e-12 * (1 + np.abs(shared).max())


# ------------------------------------------------ fused epilogue (FCN layer, f3)

@pytest.mark.parametrize("ratios,method", [([(2, 1), (2, 1)], BILINEAR), ([(4, 3), (2, 3)], BICUBIC),
                                           ([(3, 2), (3, 2)], NEAREST)])
@pytest.mark.parametrize("act", (0, 1, 2, 3))
def test_fused_matches_construction_then_library_conv1x1(orc, ratios, method, act):
    """The paper's construction (library ops) followed by torch's 1x1 convolution, bias and
    activation in float64 equals the oracle's fused layer."""
    import torch
    import torch.nn.functional as F

    rng = np.random.default_rng(61 + act + 3 * method)
    C, O = 3, 5
    x = rng.standard_normal((2, C, 9, 11))
    mix = rng.standard_normal((O, C))
    bias = rng.standard_normal(O)
    axes = []
    for r, s in ratios:
        W, K = orc.make_weights(method, r, s, 0)
        axes.append(dict(r=r, s=s, method=method, K=K, w=W))
    z = torch.from_numpy(_construction(x, axes, REFL, 0.0))
    v = F.conv2d(z, torch.from_numpy(mix).reshape(O, C, 1, 1), torch.from_numpy(bias))
    want = {0: lambda t: t, 1: F.relu, 2: lambda t: F.leaky_relu(t, 0.2),
            3: lambda t: torch.clamp(t, -0.5, 0.75)}[act](v).numpy()
    got = orc.resize_fused(x, [dict(r=r, s=s, method=method) for r, s in ratios], mix, bias, act, alpha=0.2,
                           lo=-0.5, hi=0.75, pad=REFL)
    assert got.shape == want.shape
    assert np.abs(got - want).max() <= 1e-12 * (1 + np.abs(want).max())


def test_fused_identity_mix_is_the_plain_layer(orc):
    rng = np.random.default_rng(67)
    x = rng.standard_normal((1, 4, 10, 12))
    axes = [dict(r=3, s=2, method=BICUBIC)] * 2
    z = orc.resize(x, axes, pad=CONST, pad_value=0.25)
    assert np.array_equal(orc.resize_fused(x, axes, pad=CONST, pad_value=0.25), z)
    # relu of the identity layer keeps exactly the positive outputs
    y = orc.resize_fused(x, axes, act=1, pad=CONST, pad_value=0.25)
    assert np.array_equal(y, np.where(z > 0, z, 0.0))
    # a mix that permutes channels permutes the outputs
    perm = np.eye(4)[[2, 0, 3, 1]]
    assert np.allclose(orc.resize_fused(x, axes, mix=perm, pad=CONST, pad_value=0.25), z[:, [2, 0, 3, 1]],
                       rtol=0, atol=1e-15)


# ------------------------------------------------- antialiased downscale (f4)

AA_RATIOS = [(2, 3), (1, 2), (3, 7), (2, 5), (3, 4)]


@pytest.mark.parametrize("method,mode", [(BILINEAR, "bilinear"), (BICUBIC, "bicubic")])
@pytest.mark.parametrize("pad,tpad", [(REPL, "replicate"), (REFL, "reflect"), (CONST, "constant")])
def test_antialias_matches_library_on_padded_input(orc, method, mode, pad, tpad):
    # float64 library interpolation with antialias=True at half-pixel centres equals the oracle's
    # widened, renormalised kernel wherever the library's window stays inside its input; padding the
    # input by M = m s pixels first (the library's own padding op) moves every output of the
    # original image into that interior (output o -> o + m r), which pins the extension rule too.
    # The library's antialiased bicubic uses the Keys constant a = -1/2.
    torch = pytest.importorskip("torch")
    import torch.nn.functional as TF

    rng = np.random.default_rng(61 + method + 3 * pad)
    x = rng.random((1, 2, 40, 53))
    c = 0.3
    R = 1 if method == BILINEAR else 2
    for r, s in AA_RATIOS:
        m = R + 2
        M = m * s
        xp = TF.pad(torch.from_numpy(x), (M, M, M, M), mode=tpad, **({"value": c} if tpad == "constant" else {}))
        ref = TF.interpolate(xp, scale_factor=r / s, mode=mode, align_corners=False, antialias=True,
                             recompute_scale_factor=False).numpy()
        y = orc.resize(x, [dict(r=r, s=s, method=method, align=1, antialias=1)] * 2, pad=pad, pad_value=c)
        Ho, Wo = y.shape[2:]
        sub = ref[:, :, m * r:m * r + Ho, m * r:m * r + Wo]
        assert np.abs(y - sub).max() <= 1e-13, (r, s)


def test_antialias_closed_form_half_scale_bilinear(orc):
    # paper alignment, 1/2: the hat stretched by 2 gives weights 1/4, 1/2, 1/4 at 2o - 1, 2o, 2o + 1
    rng = np.random.default_rng(67)
    x = rng.random((1, 1, 31))
    y = orc.resize(x, [dict(r=1, s=2, method=BILINEAR, antialias=1)])[0, 0]
    xe = np.concatenate([[x[0, 0, 0]], x[0, 0], [x[0, 0, -1]]])  # replicate one sample each side
    want = 0.25 * xe[0:-2:2][:len(y)] + 0.5 * xe[1:-1:2][:len(y)] + 0.25 * xe[2::2][:len(y)]
    assert np.abs(y - want).max() <= 1e-15


@pytest.mark.parametrize("method", (BILINEAR, BICUBIC))
@pytest.mark.parametrize("align", (0, 1))
def test_antialias_invariants(orc, method, align):
    rng = np.random.default_rng(71)
    x = rng.random((1, 2, 23, 29))
    for r, s in AA_RATIOS + [(3, 2), (4, 3), (1, 1), (5, 5)]:
        ax = [dict(r=r, s=s, method=method, align=align, antialias=1)] * 2
        # the weights of every output sum to one: constants are kept at every pad (the constant pad
        # with the same value)
        for pad in (REPL, CONST, REFL):
            y = orc.resize(np.full_like(x, 0.7), ax, pad=pad, pad_value=0.7)
            assert np.abs(y - 0.7).max() <= 1e-14
        # no downscale (s <= r): the widened kernel is the plain one
        plain = orc.resize(x, [dict(r=r, s=s, method=method, align=align)] * 2)
        aa = orc.resize(x, ax)
        if s <= r:
            assert np.array_equal(plain, aa)
        else:
            assert not np.allclose(plain, aa)


def test_antialias_adjoint_dot_product(orc):
    rng = np.random.default_rng(73)
    for method in (BILINEAR, BICUBIC):
        for r, s in AA_RATIOS:
            ax = [dict(r=r, s=s, method=method, align=1, antialias=1)] * 2
            for pad in (REPL, CONST, REFL):
                x = rng.standard_normal((1, 2, 19, 26))
                y = orc.resize(x, ax, pad=pad, pad_value=0.0)
                g = rng.standard_normal(y.shape)
                dx = orc.adjoint_dx(g, x.shape[2:], ax, pad=pad)
                lhs, rhs = np.vdot(y, g), np.vdot(x, dx)
                assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.abs(y).sum())
