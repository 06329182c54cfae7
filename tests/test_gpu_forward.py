"""GPU parity of the forward kernels against the FP64 oracle (through the C ABI).

Bars: nearest bit-exact; FP32 max|err| <= 2e-6 * max|x|; BF16 storage
max|err| <= 1e-2 * max|x| (oracle fed the bf16-rounded inputs); learnable
weights scale the bound by prod_a max_j sum_m |W_a[j][m]|.
"""
import numpy as np
import pytest
import torch

from paper_2203_10670_gb300 import inputs

pytestmark = pytest.mark.gpu

NEAREST, BILINEAR, BICUBIC = 0, 1, 2
REPL, CONST, REFL = 0, 1, 2
TOL = {torch.float32: 2e-6, torch.bfloat16: 1e-2}


@pytest.fixture(scope="module")
def F():
    from paper_2203_10670_gb300 import build

    build.build()
    from paper_2203_10670_gb300 import fcfs

    assert torch.cuda.is_available()
    return fcfs


def _oracle_axes(axes):
    out = []
    for a in axes:
        d = dict(r=a.r, s=a.s, method=a.method, K=a.K)
        if a.w is not None:
            d["w"] = a.w.detach().double().cpu().numpy()
        out.append(d)
    return out


def _weight_scale(axes):
    sc = 1.0
    for a in axes:
        if a.w is not None:
            sc *= float(a.w.abs().sum(-1).max())
        else:
            sc *= 1.25  # Keys weights sum to at most 1.25 in absolute value
    return sc


def check_forward(F, orc, x_cpu, axes, pad=REPL, pad_value=0.0, out_dtype=None, report=None):
    """Run the CUDA forward and compare with the oracle; returns max|err|/max|x|."""
    y = F.resize(x_cpu.cuda(), axes, pad, pad_value, out_dtype)
    torch.cuda.synchronize()
    x64 = x_cpu.double().numpy()
    learn = any(a.w is not None for a in axes)
    want = orc.resize(x64, _oracle_axes(axes), pad=pad, pad_value=pad_value, polyphase=learn)
    got = y.double().cpu().numpy()
    assert got.shape == want.shape
    if got.size == 0:
        return 0.0
    all_nearest = all(a.method == NEAREST and a.w is None for a in axes)
    if all_nearest and y.dtype == x_cpu.dtype:
        # bit-exact copy: compare in the storage type
        assert torch.equal(y.cpu(), torch.from_numpy(want).to(y.dtype)), "nearest must be bit-exact"
        return 0.0
    xmax = max(float(np.abs(x64).max()), abs(pad_value) if pad == CONST else 0.0, 1e-30)
    err = float(np.abs(got - want).max()) / xmax
    tol = TOL[y.dtype] * (_weight_scale(axes) if learn else 1.0)
    assert err <= tol, f"max|err|/max|x| = {err:.3e} > {tol:.1e}"
    if report is not None:
        report.append(err)
    return err


def test_config1_bilinear_3_2(F, orc):
    x = inputs.uniform(inputs.C1["shape"], inputs.C1["seed"])
    errs = []
    check_forward(F, orc, x, [F.Axis(3, 2, BILINEAR)] * 2, REPL, report=errs)
    for m in (NEAREST, BICUBIC):
        check_forward(F, orc, x, [F.Axis(3, 2, m)] * 2, REPL)
    print(f"c1 bilinear 3/2 max|err|/max|x| = {errs[0]:.3e}")


RATIOS_2D = [((2, 3), (2, 3)), ((4, 3), (4, 3)), ((3, 2), (3, 2)), ((5, 4), (7, 5)), ((1, 2), (2, 1)),
             ((27, 11), (2, 11)), ((1, 1), (3, 1)), ((5, 2), (3, 4))]


# width 301: rows not a multiple of 16 bytes -> gather-staged kernel;
# width 304: bulk-copy (TMA) staged persistent kernel
@pytest.mark.parametrize("width", (301, 304))
@pytest.mark.parametrize("ry,rx", RATIOS_2D)
@pytest.mark.parametrize("method", (NEAREST, BILINEAR, BICUBIC))
@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
def test_2d_ratios_methods_pads_fp32(F, orc, ry, rx, method, pad, width):
    # ragged sizes spanning several tiles in both directions
    x = inputs.uniform((2, 3, 53, width), 11 + method)
    check_forward(F, orc, x, [F.Axis(*ry, method), F.Axis(*rx, method)], pad, pad_value=0.375)


@pytest.mark.parametrize("width", (250, 256))
@pytest.mark.parametrize("method", (NEAREST, BILINEAR, BICUBIC))
@pytest.mark.parametrize("ratio", ((2, 3), (4, 3), (3, 2), (5, 4)))
@pytest.mark.parametrize("pad", (REPL, REFL))
def test_2d_bf16_storage(F, orc, method, ratio, width, pad):
    x = inputs.normal((2, 4, 67, width), 21, dtype=torch.bfloat16)
    check_forward(F, orc, x, [F.Axis(*ratio, method)] * 2, pad)


def test_bf16_constant_pad_is_rounded_to_storage(F, orc):
    # the constant of the padding is a sample of the padded input, so it takes the input's storage type
    x = inputs.normal((1, 2, 40, 64), 22, dtype=torch.bfloat16)
    c = 0.3  # not representable in bf16
    cb = float(torch.tensor(c).to(torch.bfloat16))
    y = F.resize(x.cuda(), [F.Axis(4, 3, BICUBIC)] * 2, CONST, c)
    want = orc.resize(x.double().numpy(), [dict(r=4, s=3, method=BICUBIC)] * 2, pad=CONST, pad_value=cb)
    assert np.abs(y.double().cpu().numpy() - want).max() <= 1e-2 * float(x.double().abs().max())


@pytest.mark.parametrize("din,dout", [(torch.float32, torch.bfloat16), (torch.bfloat16, torch.float32),
                                      (torch.uint8, torch.float32), (torch.uint8, torch.bfloat16)])
@pytest.mark.parametrize("width", (77, 80))
def test_mixed_storage_types(F, orc, din, dout, width):
    if din == torch.uint8:
        x = inputs.uint8_pixels((1, 3, 45, width), 5)
    else:
        x = inputs.uniform((1, 3, 45, width), 5, dtype=din)
    for method in (NEAREST, BILINEAR, BICUBIC):
        y = F.resize(x.cuda(), [F.Axis(3, 2, method), F.Axis(2, 3, method)], out_dtype=dout)
        want = orc.resize(x.double().numpy(), [dict(r=3, s=2, method=method), dict(r=2, s=3, method=method)])
        err = np.abs(y.double().cpu().numpy() - want).max() / float(x.double().abs().max())
        assert err <= TOL[dout]


@pytest.mark.parametrize("length", (1031, 1032))
@pytest.mark.parametrize("ratio", ((3, 2), (2, 3), (5, 4), (7, 5), (27, 11)))
@pytest.mark.parametrize("method", (NEAREST, BILINEAR, BICUBIC))
def test_1d(F, orc, ratio, method, length):
    x = inputs.uniform((3, 2, length), 31)
    check_forward(F, orc, x, [F.Axis(*ratio, method)], REFL)


@pytest.mark.parametrize("ratios", [((3, 2),) * 3, ((2, 3), (4, 3), (5, 4)), ((1, 2), (3, 1), (2, 11))])
@pytest.mark.parametrize("method", (NEAREST, BILINEAR, BICUBIC))
@pytest.mark.parametrize("pad", (REPL, CONST, REFL))
@pytest.mark.parametrize("width", (41, 44))
def test_3d(F, orc, ratios, method, pad, width):
    # width 44 (16-byte rows) takes the bulk-copy volume kernel, 41 the gather kernel
    x = inputs.uniform((1, 2, 19, 23, width), 41)
    check_forward(F, orc, x, [F.Axis(r, s, method) for r, s in ratios], pad, pad_value=-0.5)


@pytest.mark.parametrize("ratios", [((3, 2),) * 3, ((2, 3), (4, 3), (5, 4))])
@pytest.mark.parametrize("method", (BILINEAR, BICUBIC))
@pytest.mark.parametrize("pad", (REPL, REFL))
def test_3d_bf16_storage(F, orc, ratios, method, pad):
    x = inputs.normal((2, 2, 17, 30, 48), 42, dtype=torch.bfloat16)
    check_forward(F, orc, x, [F.Axis(r, s, method) for r, s in ratios], pad)


@pytest.mark.parametrize("ratio,method", [((3, 2), BILINEAR), ((2, 1), BILINEAR), ((4, 3), BILINEAR),
                                          ((2, 3), BILINEAR), ((3, 2), BICUBIC)])
@pytest.mark.parametrize("width", (48, 44))
@pytest.mark.parametrize("dtype", (torch.float32, torch.bfloat16))
def test_3d_register_blocked(F, orc, ratio, method, width, dtype):
    # one phase count and span on all axes: the register-blocked volume kernel (4- or 2-wide columns)
    x = inputs.uniform((2, 2, 19, 23, width), 44, dtype=dtype)
    for pad in (REPL, CONST, REFL):
        check_forward(F, orc, x, [F.Axis(*ratio, method)] * 3, pad, pad_value=0.25)


def test_3d_many_tiles(F, orc):
    # several tiles per CTA of the persistent grid, depth chunks, ragged last tiles
    x = inputs.uniform((3, 2, 37, 70, 132), 43)
    check_forward(F, orc, x, [F.Axis(3, 2, BILINEAR), F.Axis(4, 3, BICUBIC), F.Axis(5, 4, BILINEAR)], REPL)


@pytest.mark.parametrize("per_channel", (True, False))
@pytest.mark.parametrize("ratios,K", [(((5, 4), (5, 4)), 2), (((3, 2), (2, 3)), 3), (((7, 5), (4, 3)), 4)])
@pytest.mark.parametrize("pad", (REPL, CONST))
def test_learnable_weights(F, orc, per_channel, ratios, K, pad):
    C = 5
    g = torch.Generator().manual_seed(9)
    axes = []
    for r, s in ratios:
        shape = (C, r, 2 * K + 1) if per_channel else (r, 2 * K + 1)
        axes.append(F.Axis(r, s, BILINEAR, K, (torch.randn(shape, generator=g) * 0.5).cuda()))
    for width in (150, 152):
        x = inputs.normal((2, C, 37, width), 51)
        check_forward(F, orc, x, axes, pad, pad_value=0.25)


@pytest.mark.parametrize("width", (29, 28))
def test_learnable_3d(F, orc, width):
    g = torch.Generator().manual_seed(3)
    axes = [F.Axis(r, s, BILINEAR, 2, torch.randn((2, r, 5), generator=g).cuda()) for r, s in ((3, 2), (5, 4), (2, 3))]
    x = inputs.normal((1, 2, 11, 13, width), 52)
    check_forward(F, orc, x, axes, REPL)


def test_edge_cases(F, orc):
    # tiny inputs (every index is near an edge), single pixels, empty results
    for shape in ((1, 1, 1, 1), (1, 1, 2, 3), (2, 1, 1, 9), (1, 2, 5, 1), (1, 1, 3, 4), (2, 1, 1, 8), (1, 1, 7, 12)):
        for ratio in ((3, 2), (2, 3), (5, 1), (1, 1)):
            for method in (NEAREST, BILINEAR, BICUBIC):
                for pad in (REPL, CONST, REFL):
                    x = inputs.uniform(shape, 61)
                    check_forward(F, orc, x, [F.Axis(*ratio, method)] * 2, pad, pad_value=0.7)
    y = F.resize(torch.zeros((0, 3, 8, 8), device="cuda"), [F.Axis(3, 2)] * 2)
    assert y.shape == (0, 3, 12, 12)
    y = F.resize(torch.zeros((1, 1, 1, 1), device="cuda"), [F.Axis(1, 2)] * 2)
    assert y.shape == (1, 1, 0, 0)


def test_unreduced_ratio_same_result(F):
    x = inputs.uniform((1, 2, 40, 70), 71).cuda()
    for m in (NEAREST, BILINEAR, BICUBIC):
        a = F.resize(x, [F.Axis(3, 2, m)] * 2)
        b = F.resize(x, [F.Axis(6, 4, m)] * 2)
        assert torch.equal(a, b) if m == NEAREST else torch.allclose(a, b, rtol=0, atol=1e-6)


def test_host_tensors_round_trip(F, orc):
    x = inputs.uniform((1, 3, 30, 40), 81).pin_memory()
    y = F.resize(x, [F.Axis(4, 3, BICUBIC)] * 2)
    assert not y.is_cuda
    want = orc.resize(x.double().numpy(), [dict(r=4, s=3, method=BICUBIC)] * 2)
    assert np.abs(y.double().numpy() - want).max() <= 2e-6


def test_tuned_plan_same_result(F, orc):
    x = inputs.uniform((2, 3, 200, 300), 91).cuda()
    axes = [F.Axis(4, 3, BICUBIC)] * 2
    before = F.resize(x, axes)
    d = F.make_desc(x.shape, axes, 0, 0)
    y = torch.empty_like(before)
    ms, n = F.fcfs_tune_forward(d, x.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream, 2)
    assert n >= 2 and ms > 0
    after = F.resize(x, axes)
    F.fcfs_clear_plans()
    # tile shape changes the work split, never the arithmetic order of one output
    assert torch.equal(before, after)
    # and the tuned plan's output against the oracle
    xh = x.double().cpu().numpy()
    want = orc.resize(xh, [dict(r=4, s=3, method=BICUBIC)] * 2)
    assert np.abs(after.double().cpu().numpy() - want).max() <= 2e-6 * float(np.abs(xh).max())


def test_tuned_plan_same_result_3d(F, orc):
    x = inputs.uniform((1, 2, 40, 48, 64), 92).cuda()
    axes = [F.Axis(3, 2, BILINEAR)] * 3
    before = F.resize(x, axes)
    d = F.make_desc(x.shape, axes, 0, 0)
    y = torch.empty_like(before)
    ms, n = F.fcfs_tune_forward(d, x.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream, 2)
    assert n >= 2 and ms > 0
    after = F.resize(x, axes)
    F.fcfs_clear_plans()
    assert torch.equal(before, after)
    xh = x.double().cpu().numpy()
    want = orc.resize(xh, [dict(r=3, s=2, method=BILINEAR)] * 3)
    assert np.abs(after.double().cpu().numpy() - want).max() <= 2e-6 * float(np.abs(xh).max())


# ---------------------------------------------------------- full-size configs

def _sample_idx(shape, count, seed):
    rng = np.random.default_rng(seed)
    total = int(np.prod(shape))
    idx = rng.integers(0, total, count)
    # plus the first and last rows/columns of the first and last plane
    Ho, Wo = shape[-2], shape[-1]
    plane = Ho * Wo
    edges = []
    for p in (0, total // plane - 1):
        base = p * plane
        edges += [base + c for c in range(0, Wo, max(1, Wo // 512))]
        edges += [base + (Ho - 1) * Wo + c for c in range(0, Wo, max(1, Wo // 512))]
        edges += [base + r * Wo for r in range(0, Ho, max(1, Ho // 512))]
        edges += [base + r * Wo + Wo - 1 for r in range(0, Ho, max(1, Ho // 512))]
    return np.concatenate([idx, np.array(edges, dtype=np.int64)])


@pytest.mark.parametrize("ratio,method", [((2, 3), BICUBIC), ((4, 3), BICUBIC), ((3, 2), NEAREST)])
def test_config2_full_size_sampled(F, orc, ratio, method):
    x = inputs.uniform(inputs.C2["shape"], inputs.C2["seed"], device="cuda")
    axes = [F.Axis(*ratio, method)] * 2
    y = F.resize(x, axes)
    torch.cuda.synchronize()
    xh = x.cpu().double().numpy()
    idx = _sample_idx(y.shape, 200_000, 5)
    want = orc.resize_at(xh, [dict(r=ratio[0], s=ratio[1], method=method)] * 2, idx)
    got = y.reshape(-1)[torch.from_numpy(idx).cuda()].double().cpu().numpy()
    if method == NEAREST:
        assert np.array_equal(got.astype(np.float32), want.astype(np.float32))
    else:
        assert np.abs(got - want).max() <= 2e-6 * float(np.abs(xh).max())
    # bf16 variant
    yb = F.resize(x.to(torch.bfloat16), axes)
    xb = x.to(torch.bfloat16).cpu().double().numpy()
    wantb = orc.resize_at(xb, [dict(r=ratio[0], s=ratio[1], method=method)] * 2, idx)
    gotb = yb.reshape(-1)[torch.from_numpy(idx).cuda()].double().cpu().numpy()
    assert np.abs(gotb - wantb).max() <= 1e-2 * float(np.abs(xb).max())


def test_config5_large_bicubic_7_5_sampled(F, orc):
    x = inputs.uniform(inputs.C5_2D["shape"], inputs.C5_2D["seed"], device="cuda")
    axes = [F.Axis(7, 5, BICUBIC)] * 2
    y = F.resize(x, axes)
    torch.cuda.synchronize()
    assert y.shape == (1, 3, 11468, 11468)
    xh = x.cpu().double().numpy()
    idx = _sample_idx(y.shape, 100_000, 6)
    want = orc.resize_at(xh, [dict(r=7, s=5, method=BICUBIC)] * 2, idx)
    got = y.reshape(-1)[torch.from_numpy(idx).cuda()].double().cpu().numpy()
    assert np.abs(got - want).max() <= 2e-6 * float(np.abs(xh).max())


def test_config5_volume_trilinear_full(F, orc):
    x = inputs.uniform(inputs.C5_3D["shape"], inputs.C5_3D["seed"])
    errs = []
    check_forward(F, orc, x, [F.Axis(3, 2, BILINEAR)] * 3, REPL, report=errs)
    print(f"c5 trilinear 3/2 256^3 max|err|/max|x| = {errs[0]:.3e}")


def test_device_status_clean(F):
    # every bounded wait of the bulk-copy kernels completed during this module
    assert F.fcfs_device_status(clear=True) == 0
