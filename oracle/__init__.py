"""FP64 CPU oracle for FCFS (arXiv 2203.10670) -- TEST INFRASTRUCTURE ONLY.

This package is the plain, slow reference the CUDA library is checked against.
Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The library (``paper_2203_10670_gb300``) never
imports it, and it imports nothing from the library: the two share no code.

The arithmetic lives in ``fcfs_oracle.c`` (double precision, plain loops);
this module is argument marshalling around it with numpy float64 arrays.
Method and padding codes (NEAREST=0, BILINEAR=1, BICUBIC=2; REPLICATE=0,
CONSTANT=1, REFLECT=2) are the interface codes of the C ABI.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

NEAREST, BILINEAR, BICUBIC = 0, 1, 2
PAD_REPLICATE, PAD_CONSTANT, PAD_REFLECT = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fcfs_oracle.c")
_LIB = os.path.join(_HERE, "libfcfs_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP if available) into oracle/libfcfs_oracle.so."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


ALIGN_PAPER, ALIGN_HALF_PIXEL, ALIGN_FLOOR = 0, 1, 2


class _Axis(ctypes.Structure):
    _fields_ = [("r", ctypes.c_int), ("s", ctypes.c_int), ("method", ctypes.c_int),
                ("K", ctypes.c_int), ("w", ctypes.POINTER(ctypes.c_double)),
                ("w_per_channel", ctypes.c_int), ("align", ctypes.c_int), ("cubic_a", ctypes.c_double),
                ("antialias", ctypes.c_int)]


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        i, ll, d = ctypes.c_int, ctypes.c_longlong, ctypes.c_double
        P = ctypes.c_void_p
        L.orc_kernel.restype = d
        L.orc_kernel.argtypes = [i, d]
        L.orc_kernel_a.restype = d
        L.orc_kernel_a.argtypes = [i, d, d]
        L.orc_out_len.restype = ll
        L.orc_out_len.argtypes = [ll, i, i]
        L.orc_kmin.argtypes = [i, i]
        L.orc_left_offset.argtypes = [i, i]
        L.orc_num_windows.restype = ll
        L.orc_num_windows.argtypes = [ll, i]
        L.orc_ext_index.restype = ll
        L.orc_ext_index.argtypes = [ll, ll, i]
        L.orc_make_weights.argtypes = [i, i, i, i, P]
        for f in (L.orc_resize_direct, L.orc_resize_polyphase):
            f.argtypes = [i, ll, ll, P, P, i, d, P, P]
        L.orc_resize_at.argtypes = [i, i, ll, ll, P, P, i, d, P, P, ll, P]
        L.orc_adjoint_dx.argtypes = [i, ll, ll, P, P, i, P, P]
        L.orc_adjoint_dx_at.argtypes = [i, ll, ll, P, P, i, P, P, ll, P]
        L.orc_weight_grad.argtypes = [i, ll, ll, P, P, i, d, P, P, P]
        L.orc_resize_full2d.argtypes = [ll, ll, P, P, P, i, i, d, P, P]
        L.orc_adjoint_full2d.argtypes = [ll, ll, P, P, P, i, i, P, P]
        L.orc_weight_grad_full2d.argtypes = [ll, ll, P, P, i, i, d, P, P, P]
        _lib = L
    return _lib


def num_threads() -> int:
    return lib().orc_num_threads()


# ------------------------------------------------------------------ scalars

def kernel(method: int, t: float) -> float:
    """Interpolation kernel k(t): bilinear hat or Keys a=-0.5 cubic (Sec. 5.2)."""
    return lib().orc_kernel(method, float(t))


def out_len(n: int, r: int, s: int) -> int:
    return lib().orc_out_len(n, r, s)


def kmin(method: int, s: int) -> int:
    return lib().orc_kmin(method, s)


def left_offset(K: int, s: int) -> int:
    return lib().orc_left_offset(K, s)


def num_windows(n_out: int, r: int) -> int:
    return lib().orc_num_windows(n_out, r)


def ext_index(q: int, n: int, pad: int) -> int:
    return lib().orc_ext_index(q, n, pad)


def make_weights(method: int, r: int, s: int, K: int = 0):
    """Dense table W[j][m] (r x (2K+1)) and the K used; K=0 means K_min."""
    K_used = K if K else kmin(method, s)
    W = np.zeros((r, 2 * K_used + 1), dtype=np.float64)
    rc = lib().orc_make_weights(method, r, s, K, W.ctypes.data)
    if rc < 0:
        raise ValueError(f"K={K} below K_min={kmin(method, s)}")
    return W, rc


# ------------------------------------------------------------------ tensors

def _axes(axes, keep):
    """axes: list of dicts {r, s, method, K=0, w=None (array [C or 1][r][T] or [r][T]),
    align=ALIGN_PAPER, cubic_a=0 (-1/2), antialias=0 (1: widened kernel when s > r)}."""
    arr = (_Axis * len(axes))()
    for k, a in enumerate(axes):
        w = a.get("w")
        arr[k].r, arr[k].s = a["r"], a["s"]
        arr[k].method = a.get("method", BILINEAR)
        arr[k].K = a.get("K", 0)
        arr[k].align = a.get("align", ALIGN_PAPER)
        arr[k].cubic_a = float(a.get("cubic_a", 0.0))
        arr[k].antialias = int(a.get("antialias", 0))
        if w is not None:
            w = np.ascontiguousarray(w, dtype=np.float64)
            keep.append(w)
            arr[k].w = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            arr[k].w_per_channel = 1 if w.ndim == 3 else 0
            T = w.shape[-1]
            if arr[k].K == 0:
                arr[k].K = (T - 1) // 2
            assert 2 * arr[k].K + 1 == T and w.shape[-2] == a["r"]
        else:
            arr[k].w = None
            arr[k].w_per_channel = 0
    return arr


def _shapes(in_shape):
    return (ctypes.c_longlong * 3)(*(list(in_shape) + [1] * (3 - len(in_shape))))


def out_shape(in_shape, axes):
    return tuple(out_len(n, a["r"], a["s"]) for n, a in zip(in_shape, axes))


def resize(x, axes, pad=PAD_REPLICATE, pad_value=0.0, polyphase=False):
    """y = FCFS(x).  x: float64 [n, c, *spatial]; one dict per spatial axis.

    polyphase=False: fixed methods by the direct interpolation formula.
    polyphase=True : the pad/strided-conv/pixelshuffle sum with weights w (or the
                     method table when w is None)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n, c, spatial = x.shape[0], x.shape[1], x.shape[2:]
    nd = len(spatial)
    assert nd == len(axes) and 1 <= nd <= 3
    keep = []
    ax = _axes(axes, keep)
    y = np.empty((n, c) + out_shape(spatial, axes), dtype=np.float64)
    if y.size == 0:
        return y
    f = lib().orc_resize_polyphase if polyphase else lib().orc_resize_direct
    rc = f(nd, n, c, _shapes(spatial), ctypes.cast(ax, ctypes.c_void_p), pad, float(pad_value),
           x.ctypes.data, y.ctypes.data)
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return y


def resize_at(x, axes, flat_idx, pad=PAD_REPLICATE, pad_value=0.0, polyphase=False):
    """Outputs at chosen flat indices of the [n, c, *out] result."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n, c, spatial = x.shape[0], x.shape[1], x.shape[2:]
    keep = []
    ax = _axes(axes, keep)
    idx = np.ascontiguousarray(flat_idx, dtype=np.int64)
    out = np.empty(idx.shape, dtype=np.float64)
    rc = lib().orc_resize_at(1 if polyphase else 0, len(spatial), n, c, _shapes(spatial),
                             ctypes.cast(ax, ctypes.c_void_p), pad, float(pad_value),
                             x.ctypes.data, idx.ctypes.data, idx.size, out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return out


def adjoint_dx(g, in_shape, axes, pad=PAD_REPLICATE):
    """Input gradient (transposed sum with pad folding); g: [n, c, *out]."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    n, c = g.shape[0], g.shape[1]
    keep = []
    ax = _axes(axes, keep)
    dx = np.zeros((n, c) + tuple(in_shape), dtype=np.float64)
    if dx.size == 0:
        return dx
    rc = lib().orc_adjoint_dx(len(in_shape), n, c, _shapes(in_shape), ctypes.cast(ax, ctypes.c_void_p),
                              pad, g.ctypes.data, dx.ctypes.data)
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return dx


def adjoint_dx_at(g, in_shape, axes, flat_idx, pad=PAD_REPLICATE):
    """Input gradient at chosen flat indices of [n, c, *in] (gather form)."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    n, c = g.shape[0], g.shape[1]
    keep = []
    ax = _axes(axes, keep)
    idx = np.ascontiguousarray(flat_idx, dtype=np.int64)
    out = np.empty(idx.shape, dtype=np.float64)
    rc = lib().orc_adjoint_dx_at(len(in_shape), n, c, _shapes(in_shape), ctypes.cast(ax, ctypes.c_void_p),
                                 pad, g.ctypes.data, idx.ctypes.data, idx.size, out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return out


def weight_grad(x, g, axes, pad=PAD_REPLICATE, pad_value=0.0):
    """Per-axis weight gradients, each shaped like that axis's w ([C][r][T] or [r][T])."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    n, c, spatial = x.shape[0], x.shape[1], x.shape[2:]
    keep = []
    ax = _axes(axes, keep)
    outs = []
    for k, a in enumerate(axes):
        T = 2 * ax[k].K + 1
        shape = (c, a["r"], T) if ax[k].w_per_channel else (a["r"], T)
        outs.append(np.zeros(shape, dtype=np.float64))
    ptrs = (ctypes.c_void_p * 3)(*([o.ctypes.data for o in outs] + [None] * (3 - len(outs))))
    rc = lib().orc_weight_grad(len(spatial), n, c, _shapes(spatial), ctypes.cast(ax, ctypes.c_void_p),
                               pad, float(pad_value), x.ctypes.data, g.ctypes.data, ptrs)
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return outs


# ------------------------------------------------ non-separable 2D kernels

def _full_axes(axes):
    keep = []
    ax = _axes([dict(r=a["r"], s=a["s"], method=a.get("method", BILINEAR), K=a.get("K", 0)) for a in axes], keep)
    return ax


def resize_full2d(x, axes, w, pad=PAD_REPLICATE, pad_value=0.0):
    """Non-separable 2D FCFS: w [C][r_y][r_x][T_y][T_x] (per channel) or [r_y][r_x][T_y][T_x];
    axes: two dicts {r, s, K (or method for K_min)}."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    n, c, spatial = x.shape[0], x.shape[1], x.shape[2:]
    assert len(spatial) == 2 and len(axes) == 2
    ax = _full_axes(axes)
    y = np.empty((n, c) + out_shape(spatial, axes), dtype=np.float64)
    if y.size == 0:
        return y
    rc = lib().orc_resize_full2d(n, c, _shapes(spatial), ctypes.cast(ax, ctypes.c_void_p), w.ctypes.data,
                                 1 if w.ndim == 5 else 0, pad, float(pad_value), x.ctypes.data, y.ctypes.data)
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return y


def adjoint_full2d(g, in_shape, axes, w, pad=PAD_REPLICATE):
    g = np.ascontiguousarray(g, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    n, c = g.shape[0], g.shape[1]
    ax = _full_axes(axes)
    dx = np.zeros((n, c) + tuple(in_shape), dtype=np.float64)
    if dx.size == 0:
        return dx
    rc = lib().orc_adjoint_full2d(n, c, _shapes(in_shape), ctypes.cast(ax, ctypes.c_void_p), w.ctypes.data,
                                  1 if w.ndim == 5 else 0, pad, g.ctypes.data, dx.ctypes.data)
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return dx


def weight_grad_full2d(x, g, axes, per_channel, pad=PAD_REPLICATE, pad_value=0.0):
    x = np.ascontiguousarray(x, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    n, c, spatial = x.shape[0], x.shape[1], x.shape[2:]
    ax = _full_axes(axes)
    T = [2 * ax[k].K + 1 for k in range(2)]
    shape = (axes[0]["r"], axes[1]["r"], T[0], T[1])
    dw = np.zeros(((c,) + shape) if per_channel else shape, dtype=np.float64)
    rc = lib().orc_weight_grad_full2d(n, c, _shapes(spatial), ctypes.cast(ax, ctypes.c_void_p),
                                      1 if per_channel else 0, pad, float(pad_value), x.ctypes.data, g.ctypes.data,
                                      dw.ctypes.data)
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return dw


# ------------------------------------------------------- fused epilogue (FCN layer)

ACT_NONE, ACT_RELU, ACT_LEAKY_RELU, ACT_CLAMP = 0, 1, 2, 3


def resize_fused(x, axes, mix=None, bias=None, act=ACT_NONE, alpha=0.0, lo=0.0, hi=0.0, pad=PAD_REPLICATE,
                 pad_value=0.0, align=None):
    """FCFS followed by the pointwise layer that comes next in a fully convolutional
    network (Sec. 1: the resize as one layer of an FCN; Sec. 4 for the 2D layer):
        z = FCFS(x)                                  (the oracle's direct formula)
        v[n,o,p] = sum_c mix[o][c] z[n,c,p] + bias[o]  (a 1x1 convolution; mix None: v = z)
        y = act(v): none, relu max(v, 0), leaky relu (v if v >= 0 else alpha v),
                    clamp min(max(v, lo), hi).
    Float64 throughout; the channel sum is a library matrix product (one step)."""
    if align is not None:
        axes = [dict(a, align=align) for a in axes]
    # learnable taps: the strided-convolution sum with the learned weights (Sec. 3.1); fixed
    # methods: the direct interpolation formula
    z = resize(x, axes, pad=pad, pad_value=pad_value, polyphase=any(a.get("w") is not None for a in axes))
    nd = z.ndim - 2
    if mix is None:
        v = z.copy()
    else:
        mix = np.asarray(mix, dtype=np.float64)
        v = np.einsum("oc,nc...->no...", mix, z)
    if bias is not None:
        v = v + np.asarray(bias, dtype=np.float64).reshape((1, -1) + (1,) * nd)
    if act == ACT_RELU:
        v = np.maximum(v, 0.0)
    elif act == ACT_LEAKY_RELU:
        v = np.where(v >= 0.0, v, alpha * v)
    elif act == ACT_CLAMP:
        v = np.minimum(np.maximum(v, lo), hi)
    elif act != ACT_NONE:
        raise ValueError("unknown activation")
    return v


def act_derivative(v, act, alpha=0.0, lo=0.0, hi=0.0):
    """Derivative of the fused layer's activation at the pre-activation v, with the
    conventions of the common frameworks at the kinks: relu 1 for v > 0 else 0; leaky relu
    1 for v > 0 else alpha; clamp 1 for lo <= v <= hi else 0; none 1."""
    v = np.asarray(v, dtype=np.float64)
    if act == ACT_NONE:
        return np.ones_like(v)
    if act == ACT_RELU:
        return (v > 0.0).astype(np.float64)
    if act == ACT_LEAKY_RELU:
        return np.where(v > 0.0, 1.0, alpha)
    if act == ACT_CLAMP:
        return ((v >= lo) & (v <= hi)).astype(np.float64)
    raise ValueError("unknown activation")


def resize_fused_backward(x, gy, axes, mix=None, bias=None, act=ACT_NONE, alpha=0.0, lo=0.0, hi=0.0,
                          pad=PAD_REPLICATE, pad_value=0.0, align=None):
    """Gradients of the fused layer y = act(mix z + bias), z = FCFS(x), for the upstream
    gradient gy, by the chain rule step by step (float64):
        v = mix z + bias,  gv = gy act'(v),
        gmix[o][c] = sum_{n,p} gv[n,o,p] z[n,c,p],  gbias[o] = sum_{n,p} gv[n,o,p],
        gz = mix^T gv (gz = gv without a mix),
        gx = the FCFS input gradient of gz, gw = the FCFS weight gradients of gz.
    Returns (gx, gmix, gbias, gw list); gmix / gbias None where the layer has no such term."""
    if align is not None:
        axes = [dict(a, align=align) for a in axes]
    x = np.asarray(x, dtype=np.float64)
    gy = np.asarray(gy, dtype=np.float64)
    z = resize(x, axes, pad=pad, pad_value=pad_value, polyphase=any(a.get("w") is not None for a in axes))
    nd = z.ndim - 2
    if mix is None:
        v = z.copy()
    else:
        mix = np.asarray(mix, dtype=np.float64)
        v = np.einsum("oc,nc...->no...", mix, z)
    if bias is not None:
        v = v + np.asarray(bias, dtype=np.float64).reshape((1, -1) + (1,) * nd)
    gv = gy * act_derivative(v, act, alpha, lo, hi)
    axes_sum = (0,) + tuple(range(2, 2 + nd))
    gbias = gv.sum(axis=axes_sum) if bias is not None else None
    if mix is None:
        gmix, gz = None, gv
    else:
        gmix = np.einsum("nop,ncp->oc", gv.reshape(gv.shape[0], gv.shape[1], -1), z.reshape(z.shape[0], z.shape[1], -1))
        gz = np.einsum("oc,no...->nc...", mix, gv)
    gx = adjoint_dx(gz, x.shape[2:], axes, pad=pad)
    learn = [a for a in axes if a.get("w") is not None]
    gw = weight_grad(x, gz, axes, pad=pad, pad_value=pad_value) if learn else [None] * len(axes)
    return gx, gmix, gbias, gw
