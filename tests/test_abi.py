"""C-ABI checks that need no GPU: the library loads, exports every entry point
include/fcfs.h declares, computes its host-side tables like the oracle, and
rejects malformed arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_2203_10670_gb300 import build

    build.build()
    from paper_2203_10670_gb300 import _native

    return _native


def _declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(fcfs_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(native):
    lib = ctypes.CDLL(native.LIB_PATH)
    declared = _declared_functions()
    assert "fcfs_forward" in declared and "fcfs_backward" in declared
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding knows every one of them
    assert declared <= set(native.SIGNATURES), declared - set(native.SIGNATURES)


def test_every_exported_entry_point_is_declared(native):
    # the reverse direction: no fcfs_* function leaves the library undeclared
    import subprocess

    out = subprocess.run(["nm", "-D", "--defined-only", native.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = {m.group(1) for m in re.finditer(r"\sT\s(fcfs_\w+)$", out, flags=re.M)}
    assert "fcfs_forward" in exported
    undeclared = sorted(exported - _declared_functions())
    assert not undeclared, undeclared


def test_status_strings(native):
    lib = native.load()
    assert lib.fcfs_status_string(0) == b"ok"
    for code in range(-7, 0):
        assert lib.fcfs_status_string(code) not in (b"ok", b"unknown status")


RATIOS = [(3, 2), (2, 3), (4, 3), (5, 4), (7, 5), (1, 1), (2, 1), (1, 2), (5, 2), (2, 11), (27, 11)]


@pytest.mark.parametrize("method", (0, 1, 2))
@pytest.mark.parametrize("r,s", RATIOS)
def test_make_weights_matches_oracle_table(orc, native, method, r, s):
    from paper_2203_10670_gb300 import fcfs

    for extra in (0, 2):
        K = orc.kmin(method, s) + extra
        w, k_used = fcfs.fcfs_make_weights(method, r, s, K)
        want, k2 = orc.make_weights(method, r, s, K)
        assert k_used == k2 == K
        # FP64 table rounded once to FP32
        assert np.array_equal(w, want.astype(np.float32))


@pytest.mark.parametrize("method", (0, 1, 2))
@pytest.mark.parametrize("r,s", RATIOS)
def test_geometry_matches_oracle(orc, native, method, r, s):
    from paper_2203_10670_gb300 import fcfs

    for n in (0, 1, 7, 64, 1080, 8192):
        no, nw, L = fcfs.fcfs_geometry(method, r, s, 0, n)
        assert no == orc.out_len(n, r, s)
        assert nw == orc.num_windows(no, r)
        assert L == orc.left_offset(orc.kmin(method, s), s)


def test_make_weights_errors(native):
    from paper_2203_10670_gb300 import fcfs

    with pytest.raises(native.FCFSError) as e:
        fcfs.fcfs_make_weights(2, 4, 3, 2)
    assert e.value.status == native.FCFS_ERR_KERNEL_TOO_SMALL
    for bad in ((1, 0, 2), (1, 2, 0), (5, 3, 2), (1, 65, 2)):
        with pytest.raises(native.FCFSError) as e:
            fcfs.fcfs_make_weights(bad[0], bad[1], bad[2], 0)
        assert e.value.status == native.FCFS_ERR_ARG


def _desc(native, **kw):
    from paper_2203_10670_gb300 import fcfs

    ax = [fcfs.Axis(3, 2, 1), fcfs.Axis(3, 2, 1)]
    d = fcfs.make_desc((1, 1, 64, 64), ax, native.FCFS_F32, native.FCFS_F32)
    for k, v in kw.items():
        setattr(d, k, v)
    return d


BOGUS = 0x1000  # never dereferenced: every case fails validation first


@pytest.mark.parametrize("field,value,status", [
    ("ndim", 0, -1), ("ndim", 4, -1), ("n", -1, -1), ("dtype_in", 7, -1), ("dtype_out", 2, -1),
    ("pad", 3, -1), ("align", 3, -1), ("align", -1, -1), ("cubic_a", float("inf"), -1),
    ("cubic_a", float("nan"), -1),
])
def test_forward_rejects_bad_descriptor(native, field, value, status):
    lib = native.load()
    d = _desc(native, **{field: value})
    assert lib.fcfs_forward(ctypes.byref(d), BOGUS, BOGUS, None) == status
    assert lib.fcfs_last_error() != b""


def test_forward_rejects_bad_shapes_and_axes(native):
    lib = native.load()
    d = _desc(native)
    d.out_shape[0] = 97
    assert lib.fcfs_forward(ctypes.byref(d), BOGUS, BOGUS, None) == native.FCFS_ERR_ARG
    d = _desc(native)
    d.axis[1].s = 0
    assert lib.fcfs_forward(ctypes.byref(d), BOGUS, BOGUS, None) == native.FCFS_ERR_ARG
    d = _desc(native)
    d.axis[0].method, d.axis[0].K = 2, 1
    assert lib.fcfs_forward(ctypes.byref(d), BOGUS, BOGUS, None) == native.FCFS_ERR_KERNEL_TOO_SMALL
    d = _desc(native)
    assert lib.fcfs_forward(ctypes.byref(d), None, BOGUS, None) == native.FCFS_ERR_ARG
    assert lib.fcfs_forward(None, BOGUS, BOGUS, None) == native.FCFS_ERR_ARG
    d = _desc(native)
    assert lib.fcfs_forward(ctypes.byref(d), BOGUS + 1, BOGUS, None) == native.FCFS_ERR_ARG  # misaligned


def test_empty_output_enqueues_nothing(native):
    # an empty result is valid and returns before any device work
    lib = native.load()
    d = _desc(native)
    d.n = 0
    assert lib.fcfs_forward(ctypes.byref(d), None, None, None) == native.FCFS_OK
    from paper_2203_10670_gb300 import fcfs

    d = fcfs.make_desc((2, 3, 1, 1), [fcfs.Axis(1, 2, 1), fcfs.Axis(1, 2, 1)], 0, 0)
    assert tuple(d.out_shape)[:2] == (0, 0)
    assert lib.fcfs_forward(ctypes.byref(d), None, None, None) == native.FCFS_OK


def test_backward_argument_errors(native):
    lib = native.load()
    d = _desc(native)
    d.dtype_in = native.FCFS_U8
    assert lib.fcfs_backward(ctypes.byref(d), None, BOGUS, BOGUS, None, None, 0, None) == native.FCFS_ERR_UNSUPPORTED
    d = _desc(native)
    gw = (ctypes.c_void_p * 3)(BOGUS, None, None)
    # gw for an axis without learnable weights
    assert lib.fcfs_backward(ctypes.byref(d), BOGUS, BOGUS, None, ctypes.cast(gw, ctypes.c_void_p), None, 0,
                             None) == native.FCFS_ERR_ARG
    assert lib.fcfs_backward_workspace(ctypes.byref(d)) == 0


def test_nonseparable_descriptor_errors(native):
    """Validation of the non-separable 2D kernels (w2d); every case fails on the host before any device work."""
    lib = native.load()
    d = _desc(native, w2d=BOGUS, w2d_per_channel=1)
    d.ndim = 3
    d.in_shape[2] = d.out_shape[2] = 1
    d.axis[2].r = d.axis[2].s = 1
    assert lib.fcfs_forward(ctypes.byref(d), BOGUS, BOGUS, None) == native.FCFS_ERR_ARG  # 2D only
    d = _desc(native, w2d=BOGUS, w2d_per_channel=2)
    assert lib.fcfs_forward(ctypes.byref(d), BOGUS, BOGUS, None) == native.FCFS_ERR_ARG
    d = _desc(native, w2d=BOGUS + 2, w2d_per_channel=0)
    assert lib.fcfs_forward(ctypes.byref(d), BOGUS, BOGUS, None) == native.FCFS_ERR_ARG  # misaligned weights
    d = _desc(native, w2d=BOGUS, w2d_per_channel=0)
    d.axis[0].w = BOGUS
    assert lib.fcfs_forward(ctypes.byref(d), BOGUS, BOGUS, None) == native.FCFS_ERR_ARG  # per-axis and w2d
    d = _desc(native, w2d=BOGUS, w2d_per_channel=0)
    d.axis[1].K = 5  # T = 11 > FCFS_MAX_TAPS
    assert lib.fcfs_forward(ctypes.byref(d), BOGUS, BOGUS, None) == native.FCFS_ERR_UNSUPPORTED
    from paper_2203_10670_gb300 import fcfs

    d = fcfs.make_desc((1, 1, 64, 64), [fcfs.Axis(8, 1, 1, 4), fcfs.Axis(8, 1, 1, 4)], 0, 0)
    d.w2d, d.w2d_per_channel = BOGUS, 0  # 8 * 8 * 9 * 9 = 5184 kernel entries > 4096
    assert lib.fcfs_forward(ctypes.byref(d), BOGUS, BOGUS, None) == native.FCFS_ERR_UNSUPPORTED
    assert lib.fcfs_tune_forward(ctypes.byref(_desc(native, w2d=BOGUS)), BOGUS, BOGUS, None, 1, None,
                                 None) == native.FCFS_ERR_UNSUPPORTED
    d = _desc(native, w2d=BOGUS, w2d_per_channel=1)
    gw = (ctypes.c_void_p * 3)(BOGUS, BOGUS, None)  # gw[1] must stay NULL
    assert lib.fcfs_backward(ctypes.byref(d), BOGUS, BOGUS, None, ctypes.cast(gw, ctypes.c_void_p), None, 0,
                             None) == native.FCFS_ERR_ARG
    # partial-sum records: planes x chunks x (r_y r_x T_y T_x) floats, bilinear 3/2 -> T = 3
    ws = lib.fcfs_backward_workspace(ctypes.byref(d))
    assert ws > 0 and ws % (4 * 9 * 9) == 0


def test_fused_epilogue_errors(native):
    """Validation of fcfs_forward_fused; every case fails on the host before any device work."""
    lib = native.load()
    d = _desc(native)

    def run(**kw):
        e = native.fcfs_epilogue()
        e.c_out, e.mix = 4, BOGUS
        for k, v in kw.items():
            setattr(e, k, v)
        return lib.fcfs_forward_fused(ctypes.byref(d), ctypes.byref(e), BOGUS, BOGUS, None)

    assert run(c_out=0) == native.FCFS_ERR_ARG
    assert run(mix=None, c_out=2) == native.FCFS_ERR_ARG  # identity needs c_out == c (= 1)
    assert run(act=7) == native.FCFS_ERR_ARG
    assert run(act=native.FCFS_ACT_CLAMP, lo=1.0, hi=0.0) == native.FCFS_ERR_ARG
    assert run(alpha=float("nan")) == native.FCFS_ERR_ARG
    assert run(mix=BOGUS + 2) == native.FCFS_ERR_ARG  # misaligned
    assert lib.fcfs_forward_fused(ctypes.byref(d), None, BOGUS, BOGUS, None) == native.FCFS_ERR_ARG
    d = _desc(native, w2d=BOGUS)
    assert run() == native.FCFS_ERR_UNSUPPORTED
    from paper_2203_10670_gb300 import fcfs

    d = fcfs.make_desc((1, 1, 8, 8), [fcfs.Axis(32, 1, 1), fcfs.Axis(32, 1, 1)], 0, 0)
    assert run() == native.FCFS_ERR_UNSUPPORTED  # r_y r_x > 512
    d = fcfs.make_desc((1, 1, 8, 8, 8), [fcfs.Axis(2, 1, 1)] * 3, 0, 0)
    assert run() == native.FCFS_ERR_UNSUPPORTED  # 3D


def test_descriptor_cache_returns_copies(native):
    """make_desc caches descriptors by their arguments; each call gets its own copy, so changing one
    (as several tests here do) never leaks into the next call."""
    from paper_2203_10670_gb300 import fcfs

    ax = [fcfs.Axis(3, 2, 1), fcfs.Axis(4, 3, 2)]
    a = fcfs.make_desc((2, 3, 50, 60), ax, native.FCFS_F32, native.FCFS_BF16)
    a.pad, a.axis[0].r = 2, 7
    b = fcfs.make_desc((2, 3, 50, 60), ax, native.FCFS_F32, native.FCFS_BF16)
    assert (b.pad, b.axis[0].r, b.axis[1].s, b.out_shape[0], b.out_shape[1]) == (0, 3, 3, 75, 80)
    c = fcfs.make_desc((2, 3, 50, 60), ax, native.FCFS_F32, native.FCFS_BF16, pad=1, pad_value=0.5)
    assert (c.pad, c.pad_value) == (1, 0.5) and b.pad == 0


def test_binding_argument_checks_for_the_new_layers():
    """resize_full2d / resize_fused validate their tensors before any device work."""
    import torch

    from paper_2203_10670_gb300 import fcfs

    x = torch.zeros(1, 3, 8, 8)
    ax = [fcfs.Axis(2, 1, 1), fcfs.Axis(2, 1, 1)]
    with pytest.raises(ValueError):  # weights must live on the device
        fcfs.make_desc_full2d(x.shape, ax, torch.zeros(3, 2, 2, 3, 3), 0, 0)
    with pytest.raises(ValueError):  # a non-separable layer has two spatial axes
        fcfs.make_desc_full2d((1, 3, 8, 8, 8), ax + [fcfs.Axis(2, 1, 1)], torch.zeros(2, 2, 3, 3), 0, 0)
    with pytest.raises(ValueError):  # the mix must live on the device
        fcfs.resize_fused(x, ax, mix=torch.zeros(4, 3))


def test_fused_backward_host_checks(native):
    """fcfs_backward_fused_workspace and the argument checks of fcfs_backward_fused: every case here is
    decided on the host before any device work (the pointers are never dereferenced)."""
    from paper_2203_10670_gb300 import fcfs

    lib = native.load()
    d = fcfs.make_desc((2, 3, 16, 20), [fcfs.Axis(2, 1, 1)] * 2, native.FCFS_F32, native.FCFS_F32)

    def epi(**kw):
        e = native.fcfs_epilogue()
        e.c_out, e.mix, e.bias, e.act = 5, BOGUS, BOGUS, native.FCFS_ACT_RELU
        for k, v in kw.items():
            setattr(e, k, v)
        return e

    e = epi()
    need = lib.fcfs_backward_fused_workspace(ctypes.byref(d), ctypes.byref(e))
    # the recomputed outputs (3 channels) and the activation gradient (5), FP32 at 32 x 40 pixels, at least
    assert need >= 2 * 32 * 40 * (3 + 5) * 4
    assert lib.fcfs_backward_fused_workspace(ctypes.byref(d), ctypes.byref(epi(c_out=0))) == 0
    assert lib.fcfs_backward_fused_workspace(ctypes.byref(d), ctypes.byref(epi(mix=None))) == 0  # 5 != 3
    d8 = fcfs.make_desc((2, 3, 16, 20), [fcfs.Axis(2, 1, 1)] * 2, native.FCFS_U8, native.FCFS_F32)
    assert lib.fcfs_backward_fused_workspace(ctypes.byref(d8), ctypes.byref(e)) == 0

    def run(e, gx=BOGUS, gmix=None, gbias=None, ws=BOGUS, nbytes=need):
        return lib.fcfs_backward_fused(ctypes.byref(d), ctypes.byref(e), BOGUS, BOGUS, gx, gmix, gbias, None, ws,
                                       nbytes, None)

    assert run(e, ws=None) == native.FCFS_ERR_ARG
    assert run(e, nbytes=need - 1) == native.FCFS_ERR_ARG
    assert run(e, ws=BOGUS + 16) == native.FCFS_ERR_ARG  # workspace not 256-byte aligned
    assert run(epi(mix=None, c_out=3), gmix=BOGUS) == native.FCFS_ERR_ARG  # no mix, no mix gradient
    assert run(epi(bias=None), gbias=BOGUS) == native.FCFS_ERR_ARG
    assert run(e, gx=None) == native.FCFS_OK  # nothing asked for: nothing enqueued
