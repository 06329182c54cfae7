"""Python binding of libfcfs: FCFS (arXiv 2203.10670) on GB300.

The C entry points keep their names here (``fcfs_make_weights``,
``fcfs_geometry``, ``fcfs_forward``, ``fcfs_backward``,
``fcfs_backward_workspace``, ``fcfs_tune_forward``) and take the same
arguments.  ``resize`` / ``resize_backward`` / ``FCFSFunction`` / ``FCFS`` are
thin torch-tensor wrappers around them: they build the descriptor, allocate
outputs with torch and pass pointers and the current stream.  Every step of
the layer runs in the CUDA kernels of libfcfs; nothing here computes.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import torch

from . import _native as N
from ._native import (FCFS_ALIGN_FLOOR, FCFS_ALIGN_HALF_PIXEL, FCFS_ALIGN_PAPER, FCFS_BF16, FCFS_BICUBIC,
                      FCFS_BILINEAR, FCFS_F32, FCFS_NEAREST, FCFS_PAD_CONSTANT, FCFS_PAD_REFLECT, FCFS_PAD_REPLICATE,
                      FCFS_U8, FCFSError, check)

NEAREST, BILINEAR, BICUBIC = FCFS_NEAREST, FCFS_BILINEAR, FCFS_BICUBIC
PAD_REPLICATE, PAD_CONSTANT, PAD_REFLECT = FCFS_PAD_REPLICATE, FCFS_PAD_CONSTANT, FCFS_PAD_REFLECT
ALIGN_PAPER, ALIGN_HALF_PIXEL, ALIGN_FLOOR = FCFS_ALIGN_PAPER, FCFS_ALIGN_HALF_PIXEL, FCFS_ALIGN_FLOOR

_DT = {torch.float32: FCFS_F32, torch.bfloat16: FCFS_BF16, torch.uint8: FCFS_U8}
_TD = {FCFS_F32: torch.float32, FCFS_BF16: torch.bfloat16, FCFS_U8: torch.uint8}


@dataclass
class Axis:
    """One spatial axis: scale r/s, fixed `method` (w=None) or learnable taps w
    (float32 CUDA tensor [C, r, 2K+1] per channel or [r, 2K+1] shared)."""
    r: int
    s: int
    method: int = BILINEAR
    K: int = 0
    w: Optional[torch.Tensor] = None


# ----------------------------------------------------------- raw entry points

def fcfs_make_weights(method: int, r: int, s: int, K: int = 0):
    """The FP32 weight table W[j][m] (r x (2K+1)) and the K used (K=0 -> K_min)."""
    lib = N.load()
    k_out = ctypes.c_int(0)
    check(lib.fcfs_make_weights(method, r, s, K, None, ctypes.byref(k_out)), "fcfs_make_weights")
    w = np.zeros((r, 2 * k_out.value + 1), dtype=np.float32)
    check(lib.fcfs_make_weights(method, r, s, K, w.ctypes.data, ctypes.byref(k_out)), "fcfs_make_weights")
    return w, k_out.value


def fcfs_geometry(method: int, r: int, s: int, K: int, n_in: int):
    """(n_out, n_windows, left_offset) of one axis."""
    lib = N.load()
    no, nw, lo = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_int()
    check(lib.fcfs_geometry(method, r, s, K, n_in, ctypes.byref(no), ctypes.byref(nw), ctypes.byref(lo)),
          "fcfs_geometry")
    return no.value, nw.value, lo.value


def fcfs_forward(desc: N.fcfs_desc, x_ptr: int, y_ptr: int, stream: int = 0) -> None:
    check(N.load().fcfs_forward(ctypes.byref(desc), x_ptr, y_ptr, stream), "fcfs_forward")


def fcfs_backward_workspace(desc: N.fcfs_desc) -> int:
    return int(N.load().fcfs_backward_workspace(ctypes.byref(desc)))


def fcfs_backward(desc, x_ptr, gy_ptr, gx_ptr, gw_ptrs, ws_ptr, ws_bytes, stream=0) -> None:
    arr = None
    if gw_ptrs is not None:
        arr = (ctypes.c_void_p * 3)(*(list(gw_ptrs) + [None] * (3 - len(gw_ptrs))))
    check(N.load().fcfs_backward(ctypes.byref(desc), x_ptr, gy_ptr, gx_ptr,
                                 ctypes.cast(arr, ctypes.c_void_p) if arr is not None else None,
                                 ws_ptr, ws_bytes, stream), "fcfs_backward")


def fcfs_backward_noalloc(desc, x_ptr, gy_ptr, gx_ptr, gw_ptrs, stream=0) -> None:
    """fcfs_backward with the library's built-in scratch area instead of a workspace."""
    arr = None
    if gw_ptrs is not None:
        arr = (ctypes.c_void_p * 3)(*(list(gw_ptrs) + [None] * (3 - len(gw_ptrs))))
    check(N.load().fcfs_backward_noalloc(ctypes.byref(desc), x_ptr, gy_ptr, gx_ptr,
                                         ctypes.cast(arr, ctypes.c_void_p) if arr is not None else None,
                                         stream), "fcfs_backward_noalloc")


def fcfs_tune_forward(desc, x_ptr, y_ptr, stream=0, reps=3):
    """Time the candidate tile shapes and keep the fastest for this key."""
    ms, n = ctypes.c_float(), ctypes.c_int()
    check(N.load().fcfs_tune_forward(ctypes.byref(desc), x_ptr, y_ptr, stream, reps, ctypes.byref(ms),
                                     ctypes.byref(n)), "fcfs_tune_forward")
    return ms.value, n.value


def fcfs_clear_plans() -> None:
    N.load().fcfs_clear_plans()


def fcfs_plan_count() -> int:
    """Plans in the process-wide cache (those tuned here, plus any loaded from FCFS_TUNE_CACHE)."""
    return int(N.load().fcfs_plan_count())


def fcfs_device_status(clear: bool = False) -> int:
    """Device status word (0 = every bounded wait completed); synchronizes."""
    v = N.load().fcfs_device_status(1 if clear else 0)
    if v < 0:
        check(v, "fcfs_device_status")
    return v


# ------------------------------------------------------------- descriptors

def out_len(n: int, r: int, s: int) -> int:
    return (n * r) // s


_DESC_CACHE: "dict" = {}
_DESC_CACHE_MAX = 256


def make_desc(shape: Sequence[int], axes: Sequence[Axis], dtype_in: int, dtype_out: int,
              pad: int = PAD_REPLICATE, pad_value: float = 0.0, align: int = ALIGN_PAPER,
              cubic_a: float = 0.0, antialias: bool = False) -> N.fcfs_desc:
    """Descriptor for an input of shape [n, c, *spatial] (spatial outermost first).
    align / cubic_a / antialias: sample alignment, Keys parameter and antialiased downscale of the fixed methods
    (ALIGN_PAPER and 0 = the paper's -0.5 by default).

    Descriptors are cached by their arguments (a learnable axis by its weight
    tensor's address and shape); each call returns its own copy."""
    key = (tuple(int(v) for v in shape),
           tuple((a.r, a.s, a.method, a.K, None if a.w is None else (a.w.data_ptr(), tuple(a.w.shape), a.w.dtype,
                                                                      a.w.is_cuda, a.w.is_contiguous()))
                 for a in axes),
           dtype_in, dtype_out, pad, float(pad_value), int(align), float(cubic_a), int(bool(antialias)))
    hit = _DESC_CACHE.get(key)
    if hit is not None:
        return N.fcfs_desc.from_buffer_copy(hit)
    d = _build_desc(shape, axes, dtype_in, dtype_out, pad, pad_value, align, cubic_a, antialias)
    if len(_DESC_CACHE) >= _DESC_CACHE_MAX:
        _DESC_CACHE.clear()
    _DESC_CACHE[key] = N.fcfs_desc.from_buffer_copy(d)
    return d


def _build_desc(shape, axes, dtype_in, dtype_out, pad, pad_value, align, cubic_a, antialias=False) -> N.fcfs_desc:
    nd = len(shape) - 2
    if nd != len(axes) or not 1 <= nd <= 3:
        raise ValueError(f"{len(axes)} axes for a tensor with {nd} spatial dims")
    d = N.fcfs_desc()
    d.ndim = nd
    d.n, d.c = int(shape[0]), int(shape[1])
    for a, ax in enumerate(axes):
        d.in_shape[a] = int(shape[2 + a])
        d.out_shape[a] = out_len(int(shape[2 + a]), ax.r, ax.s)
        d.axis[a].r, d.axis[a].s = ax.r, ax.s
        d.axis[a].K, d.axis[a].method = ax.K, ax.method
        if ax.w is not None:
            w = ax.w
            if w.dtype != torch.float32 or not w.is_cuda or not w.is_contiguous():
                raise ValueError("learnable weights must be contiguous float32 CUDA tensors")
            if w.shape[-2] != ax.r:
                raise ValueError("weights must have r rows")
            T = w.shape[-1]
            d.axis[a].K = ax.K if ax.K else (T - 1) // 2
            if 2 * d.axis[a].K + 1 != T:
                raise ValueError("weights must have 2K+1 taps")
            d.axis[a].w = w.data_ptr()
            d.axis[a].w_per_channel = 1 if w.dim() == 3 else 0
        else:
            d.axis[a].w = None
            d.axis[a].w_per_channel = 0
    d.dtype_in, d.dtype_out = dtype_in, dtype_out
    d.pad, d.pad_value = pad, float(pad_value)
    d.align = int(align)
    d.cubic_a = float(cubic_a)
    d.antialias = 1 if antialias else 0
    return d


def out_shape(shape: Sequence[int], axes: Sequence[Axis]):
    return tuple(shape[:2]) + tuple(out_len(n, a.r, a.s) for n, a in zip(shape[2:], axes))


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


# ------------------------------------------------------------ tensor level

def resize(x: torch.Tensor, axes: Sequence[Axis], pad: int = PAD_REPLICATE, pad_value: float = 0.0,
           out_dtype: Optional[torch.dtype] = None, out: Optional[torch.Tensor] = None, align: int = ALIGN_PAPER,
           cubic_a: float = 0.0, antialias: bool = False) -> torch.Tensor:
    """y = FCFS(x) for x [n, c, *spatial] (float32, bfloat16 or uint8).

    A CUDA tensor is processed on its device and current stream.  A host tensor
    is copied to the current CUDA device, resized there, and the result copied
    back to host memory (pinned inputs make both copies asynchronous)."""
    if not x.is_cuda:
        dev = torch.device("cuda", torch.cuda.current_device())
        y = resize(x.to(dev, non_blocking=True), axes, pad, pad_value, out_dtype, align=align, cubic_a=cubic_a,
                   antialias=antialias)
        if out is not None:
            out.copy_(y)
            return out
        return y.cpu()
    if out_dtype is None:
        out_dtype = torch.float32 if x.dtype == torch.uint8 else x.dtype
    x = x.contiguous()
    d = make_desc(x.shape, axes, _DT[x.dtype], _DT[out_dtype], pad, pad_value, align, cubic_a, antialias)
    oshape = out_shape(x.shape, axes)
    if out is None:
        out = torch.empty(oshape, dtype=out_dtype, device=x.device)
    elif tuple(out.shape) != oshape or out.dtype != out_dtype or not out.is_contiguous():
        raise ValueError("out has the wrong shape, dtype or layout")
    fcfs_forward(d, x.data_ptr(), out.data_ptr(), _stream(x.device))
    return out


def resize_backward(x: Optional[torch.Tensor], gy: torch.Tensor, axes: Sequence[Axis], pad: int = PAD_REPLICATE,
                    pad_value: float = 0.0, in_shape=None, in_dtype=None, need_dx: bool = True,
                    need_dw: Sequence[bool] = (), align: int = ALIGN_PAPER, cubic_a: float = 0.0,
                    antialias: bool = False):
    """(gx, [gw per axis]) of the FCFS forward for upstream gradient gy."""
    if in_shape is None:
        in_shape = tuple(x.shape)
    if in_dtype is None:
        in_dtype = x.dtype
    gy = gy.contiguous()
    d = make_desc(in_shape, axes, _DT[in_dtype], _DT[gy.dtype], pad, pad_value, align, cubic_a, antialias)
    dev = gy.device
    gx = torch.empty(in_shape, dtype=in_dtype, device=dev) if need_dx else None
    gws, ptrs = [], []
    for a, ax in enumerate(axes):
        want = bool(need_dw[a]) if a < len(need_dw) else False
        if want and ax.w is not None:
            g = torch.empty_like(ax.w)
            gws.append(g)
            ptrs.append(g.data_ptr())
        else:
            gws.append(None)
            ptrs.append(None)
    ws_bytes = fcfs_backward_workspace(d) if any(p is not None for p in ptrs) else 0
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=dev)
    fcfs_backward(d, x.data_ptr() if x is not None else None, gy.data_ptr(),
                  gx.data_ptr() if gx is not None else None, ptrs, ws.data_ptr(), ws_bytes, _stream(dev))
    return gx, gws


class FCFSFunction(torch.autograd.Function):
    """Differentiable FCFS: hand-written forward and backward kernels of libfcfs."""

    @staticmethod
    def forward(ctx, x, spec, *weights):
        axes = [Axis(a.r, a.s, a.method, a.K, w) for a, w in zip(spec["axes"], weights)]
        y = resize(x, axes, spec["pad"], spec["pad_value"], spec.get("out_dtype"), align=spec.get("align", ALIGN_PAPER),
                   cubic_a=spec.get("cubic_a", 0.0), antialias=spec.get("antialias", False))
        ctx.spec = spec
        ctx.save_for_backward(x, *[w if w is not None else torch.empty(0) for w in weights])
        ctx.has_w = [w is not None for w in weights]
        return y

    @staticmethod
    def backward(ctx, gy):
        x, *ws = ctx.saved_tensors
        spec = ctx.spec
        axes = [Axis(a.r, a.s, a.method, a.K, w if h else None) for a, w, h in zip(spec["axes"], ws, ctx.has_w)]
        need_w = [h and ctx.needs_input_grad[2 + i] for i, h in enumerate(ctx.has_w)]
        gx, gws = resize_backward(x if any(need_w) else None, gy.to(spec.get("out_dtype") or x.dtype), axes,
                                  spec["pad"], spec["pad_value"], in_shape=tuple(x.shape), in_dtype=x.dtype,
                                  need_dx=ctx.needs_input_grad[0], need_dw=need_w,
                                  align=spec.get("align", ALIGN_PAPER), cubic_a=spec.get("cubic_a", 0.0),
                                  antialias=spec.get("antialias", False))
        return (gx, None, *gws)


class FCFS(torch.nn.Module):
    """FCFS layer (Sec. 3.1 / Sec. 4): depthwise, separable per spatial axis.

    ratios: one (r, s) per spatial axis.  learnable=True gives each axis
    per-channel taps [C, r, 2K+1] initialised to the method's table."""

    def __init__(self, channels: int, ratios, method: int = BILINEAR, pad: int = PAD_REPLICATE,
                 pad_value: float = 0.0, learnable: bool = False, K: int = 0, out_dtype=None,
                 align: int = ALIGN_PAPER, cubic_a: float = 0.0, antialias: bool = False):
        super().__init__()
        self.ratios = [tuple(rs) for rs in ratios]
        self.method, self.pad, self.pad_value, self.out_dtype = method, pad, pad_value, out_dtype
        self.align, self.cubic_a = align, cubic_a  # fixed-method sampling (learnable taps ignore it)
        self.antialias = antialias
        self.weights = torch.nn.ParameterList()
        self.Ks = []
        for r, s in self.ratios:
            w, k = fcfs_make_weights(method, r, s, K)
            self.Ks.append(k)
            if learnable:
                self.weights.append(torch.nn.Parameter(torch.from_numpy(np.tile(w[None], (channels, 1, 1)))))
        self.learnable = learnable

    def forward(self, x):
        spec = {"axes": [Axis(r, s, self.method, k) for (r, s), k in zip(self.ratios, self.Ks)],
                "pad": self.pad, "pad_value": self.pad_value, "out_dtype": self.out_dtype,
                "align": self.align, "cubic_a": self.cubic_a, "antialias": self.antialias}
        ws = [w.contiguous() for w in self.weights] if self.learnable else [None] * len(self.ratios)
        return FCFSFunction.apply(x, spec, *ws)


# ------------------------------------------- fused pointwise layer (FCN)

ACT_NONE, ACT_RELU, ACT_LEAKY_RELU, ACT_CLAMP = (N.FCFS_ACT_NONE, N.FCFS_ACT_RELU, N.FCFS_ACT_LEAKY_RELU,
                                                 N.FCFS_ACT_CLAMP)


def fcfs_forward_fused(desc: N.fcfs_desc, epi: N.fcfs_epilogue, x_ptr: int, y_ptr: int, stream: int = 0) -> None:
    check(N.load().fcfs_forward_fused(ctypes.byref(desc), ctypes.byref(epi), x_ptr, y_ptr, stream),
          "fcfs_forward_fused")


def fcfs_backward_fused_workspace(desc: N.fcfs_desc, epi: N.fcfs_epilogue) -> int:
    return int(N.load().fcfs_backward_fused_workspace(ctypes.byref(desc), ctypes.byref(epi)))


def fcfs_backward_fused(desc, epi, x_ptr, gy_ptr, gx_ptr, gmix_ptr, gbias_ptr, gw_ptrs, ws_ptr, ws_bytes,
                        stream=0) -> None:
    arr = None
    if gw_ptrs is not None:
        arr = (ctypes.c_void_p * 3)(*(list(gw_ptrs) + [None] * (3 - len(gw_ptrs))))
    check(N.load().fcfs_backward_fused(ctypes.byref(desc), ctypes.byref(epi), x_ptr, gy_ptr, gx_ptr, gmix_ptr,
                                       gbias_ptr, ctypes.cast(arr, ctypes.c_void_p) if arr is not None else None,
                                       ws_ptr, ws_bytes, stream), "fcfs_backward_fused")


def _fused_epilogue(c: int, mix, bias, act, alpha, lo, hi) -> N.fcfs_epilogue:
    e = N.fcfs_epilogue()
    for name, t in (("mix", mix), ("bias", bias)):
        if t is not None and (t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    e.c_out = int(mix.shape[0]) if mix is not None else int(c)
    if mix is not None and tuple(mix.shape) != (e.c_out, c):
        raise ValueError("mix must be [c_out, c]")
    if bias is not None and tuple(bias.shape) != (e.c_out,):
        raise ValueError("bias must be [c_out]")
    e.mix = mix.data_ptr() if mix is not None else None
    e.bias = bias.data_ptr() if bias is not None else None
    e.act, e.alpha, e.lo, e.hi = int(act), float(alpha), float(lo), float(hi)
    return e


def resize_fused_backward(x: torch.Tensor, gy: torch.Tensor, axes: Sequence[Axis], mix: Optional[torch.Tensor] = None,
                          bias: Optional[torch.Tensor] = None, act: int = ACT_NONE, alpha: float = 0.0,
                          lo: float = 0.0, hi: float = 0.0, pad: int = PAD_REPLICATE, pad_value: float = 0.0,
                          align: int = ALIGN_PAPER, cubic_a: float = 0.0, need_dx: bool = True,
                          need_dmix: bool = False, need_dbias: bool = False, need_dw: Sequence[bool] = ()):
    """(gx, gmix, gbias, [gw per axis]) of y = act(mix @ FCFS(x) + bias) for the upstream gradient gy
    (fcfs_backward_fused); entries not asked for are None."""
    x = x.contiguous()
    gy = gy.contiguous()
    d = make_desc(x.shape, axes, _DT[x.dtype], _DT[gy.dtype], pad, pad_value, align, cubic_a)
    e = _fused_epilogue(x.shape[1], mix, bias, act, alpha, lo, hi)
    dev = x.device
    gx = torch.empty_like(x) if need_dx else None
    gmix = torch.empty_like(mix) if need_dmix and mix is not None else None
    gbias = torch.empty_like(bias) if need_dbias and bias is not None else None
    gws, ptrs = [], []
    for a, ax in enumerate(axes):
        want = bool(need_dw[a]) if a < len(need_dw) else False
        g = torch.empty_like(ax.w) if want and ax.w is not None else None
        gws.append(g)
        ptrs.append(g.data_ptr() if g is not None else None)
    ws_bytes = fcfs_backward_fused_workspace(d, e)
    if ws_bytes == 0:  # the descriptor or epilogue was refused (the library's message says why)
        raise N.FCFSError(N.FCFS_ERR_ARG, "fcfs_backward_fused_workspace")
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=dev)
    fcfs_backward_fused(d, e, x.data_ptr(), gy.data_ptr(), gx.data_ptr() if gx is not None else None,
                        gmix.data_ptr() if gmix is not None else None, gbias.data_ptr() if gbias is not None else None,
                        ptrs, ws.data_ptr(), ws_bytes, _stream(dev))
    return gx, gmix, gbias, gws


def resize_fused(x: torch.Tensor, axes: Sequence[Axis], mix: Optional[torch.Tensor] = None,
                 bias: Optional[torch.Tensor] = None, act: int = ACT_NONE, alpha: float = 0.0, lo: float = 0.0,
                 hi: float = 0.0, pad: int = PAD_REPLICATE, pad_value: float = 0.0,
                 out_dtype: Optional[torch.dtype] = None, align: int = ALIGN_PAPER, cubic_a: float = 0.0,
                 antialias: bool = False,
                 out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """y = act(mix @ FCFS(x) + bias) over channels, in one kernel (x [n, c, H, W] on a CUDA device;
    mix [c_out, c] float32 or None for the identity; bias [c_out] or None)."""
    if out_dtype is None:
        out_dtype = out.dtype if out is not None else torch.float32 if x.dtype == torch.uint8 else x.dtype
    x = x.contiguous()
    d = make_desc(x.shape, axes, _DT[x.dtype], _DT[out_dtype], pad, pad_value, align, cubic_a, antialias)
    e = _fused_epilogue(x.shape[1], mix, bias, act, alpha, lo, hi)
    oshape = (x.shape[0], e.c_out) + out_shape(x.shape, axes)[2:]
    if out is None:
        out = torch.empty(oshape, dtype=out_dtype, device=x.device)
    elif tuple(out.shape) != oshape or out.dtype != out_dtype or not out.is_contiguous():
        raise ValueError("out has the wrong shape, dtype or layout")
    fcfs_forward_fused(d, e, x.data_ptr(), out.data_ptr(), _stream(x.device))
    return out


class FusedFunction(torch.autograd.Function):
    """Differentiable fused layer y = act(mix @ FCFS(x) + bias): fcfs_forward_fused and
    fcfs_backward_fused (gradients of x, mix, bias and the learnable taps)."""

    @staticmethod
    def forward(ctx, x, spec, mix, bias, *weights):
        axes = [Axis(a.r, a.s, a.method, a.K, w) for a, w in zip(spec["axes"], weights)]
        y = resize_fused(x, axes, mix, bias, spec["act"], spec["alpha"], spec["lo"], spec["hi"], spec["pad"],
                         spec["pad_value"], out_dtype=spec.get("out_dtype"))
        ctx.spec = spec
        ctx.has = [mix is not None, bias is not None] + [w is not None for w in weights]
        ctx.save_for_backward(x, *[t if t is not None else torch.empty(0) for t in (mix, bias, *weights)])
        return y

    @staticmethod
    def backward(ctx, gy):
        x, mix, bias, *ws = ctx.saved_tensors
        spec = ctx.spec
        mix = mix if ctx.has[0] else None
        bias = bias if ctx.has[1] else None
        axes = [Axis(a.r, a.s, a.method, a.K, w if h else None) for a, w, h in zip(spec["axes"], ws, ctx.has[2:])]
        need_w = [h and ctx.needs_input_grad[4 + i] for i, h in enumerate(ctx.has[2:])]
        gx, gmix, gbias, gws = resize_fused_backward(
            x, gy.to(spec.get("out_dtype") or x.dtype), axes, mix, bias, spec["act"], spec["alpha"], spec["lo"],
            spec["hi"], spec["pad"], spec["pad_value"], need_dx=ctx.needs_input_grad[0],
            need_dmix=mix is not None and ctx.needs_input_grad[2],
            need_dbias=bias is not None and ctx.needs_input_grad[3], need_dw=need_w)
        return (gx, None, gmix, gbias, *gws)


class FCFSFused(torch.nn.Module):
    """FCFS followed by a 1x1 convolution, bias and activation in one layer (the resize as a
    layer of a fully convolutional network), trained through FusedFunction."""

    def __init__(self, channels: int, out_channels: int, ratios, method: int = BILINEAR, act: int = ACT_RELU,
                 alpha: float = 0.0, lo: float = 0.0, hi: float = 0.0, pad: int = PAD_REPLICATE,
                 pad_value: float = 0.0, learnable: bool = False, K: int = 0, bias: bool = True, out_dtype=None):
        super().__init__()
        self.ratios = [tuple(rs) for rs in ratios]
        self.method, self.act, self.alpha, self.lo, self.hi = method, act, alpha, lo, hi
        self.pad, self.pad_value, self.out_dtype = pad, pad_value, out_dtype
        self.mix = torch.nn.Parameter(torch.randn(out_channels, channels) / math.sqrt(channels))
        self.bias = torch.nn.Parameter(torch.zeros(out_channels)) if bias else None
        self.weights = torch.nn.ParameterList()
        self.Ks = []
        for r, s in self.ratios:
            w, k = fcfs_make_weights(method, r, s, K)
            self.Ks.append(k)
            if learnable:
                self.weights.append(torch.nn.Parameter(torch.from_numpy(np.tile(w[None], (channels, 1, 1)))))
        self.learnable = learnable

    def forward(self, x):
        spec = {"axes": [Axis(r, s, self.method, k) for (r, s), k in zip(self.ratios, self.Ks)],
                "act": self.act, "alpha": self.alpha, "lo": self.lo, "hi": self.hi, "pad": self.pad,
                "pad_value": self.pad_value, "out_dtype": self.out_dtype}
        ws = [w.contiguous() for w in self.weights] if self.learnable else [None] * len(self.ratios)
        return FusedFunction.apply(x, spec, self.mix.contiguous(), self.bias, *ws)


# ------------------------------------------------- non-separable 2D kernels

def _full2d_axes(axes: Sequence[Axis], w2d: torch.Tensor):
    if len(axes) != 2:
        raise ValueError("non-separable kernels take two spatial axes")
    if w2d.dtype != torch.float32 or not w2d.is_cuda or not w2d.is_contiguous() or w2d.dim() not in (4, 5):
        raise ValueError("w2d must be a contiguous float32 CUDA tensor [C, r_y, r_x, T_y, T_x] or [r_y, r_x, T_y, T_x]")
    ry, rx, Ty, Tx = w2d.shape[-4:]
    if (ry, rx) != (axes[0].r, axes[1].r) or Ty % 2 == 0 or Tx % 2 == 0:
        raise ValueError("w2d must have r_y x r_x phases of odd T_y x T_x taps")
    return [Axis(axes[0].r, axes[0].s, axes[0].method, (Ty - 1) // 2),
            Axis(axes[1].r, axes[1].s, axes[1].method, (Tx - 1) // 2)]


def make_desc_full2d(shape: Sequence[int], axes: Sequence[Axis], w2d: torch.Tensor, dtype_in: int, dtype_out: int,
                     pad: int = PAD_REPLICATE, pad_value: float = 0.0) -> N.fcfs_desc:
    """Descriptor of the non-separable 2D layer: axes give r and s; K follows from w2d's taps."""
    d = make_desc(shape, _full2d_axes(axes, w2d), dtype_in, dtype_out, pad, pad_value)
    d.w2d = w2d.data_ptr()
    d.w2d_per_channel = 1 if w2d.dim() == 5 else 0
    return d


def resize_full2d(x: torch.Tensor, axes: Sequence[Axis], w2d: torch.Tensor, pad: int = PAD_REPLICATE,
                  pad_value: float = 0.0, out_dtype: Optional[torch.dtype] = None,
                  out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """y = FCFS(x) with one general T_y x T_x kernel per phase pair (x [n, c, H, W] on a CUDA device)."""
    if out_dtype is None:
        out_dtype = out.dtype if out is not None else torch.float32 if x.dtype == torch.uint8 else x.dtype
    x = x.contiguous()
    d = make_desc_full2d(x.shape, axes, w2d, _DT[x.dtype], _DT[out_dtype], pad, pad_value)
    oshape = out_shape(x.shape, axes)
    if out is None:
        out = torch.empty(oshape, dtype=out_dtype, device=x.device)
    elif tuple(out.shape) != oshape or out.dtype != out_dtype or not out.is_contiguous():
        raise ValueError("out has the wrong shape, dtype or layout")
    fcfs_forward(d, x.data_ptr(), out.data_ptr(), _stream(x.device))
    return out


def resize_full2d_backward(x: Optional[torch.Tensor], gy: torch.Tensor, axes: Sequence[Axis], w2d: torch.Tensor,
                           pad: int = PAD_REPLICATE, pad_value: float = 0.0, in_shape=None, in_dtype=None,
                           need_dx: bool = True, need_dw: bool = True):
    """(gx, gw2d) of resize_full2d for upstream gradient gy."""
    if in_shape is None:
        in_shape = tuple(x.shape)
    if in_dtype is None:
        in_dtype = x.dtype
    gy = gy.contiguous()
    d = make_desc_full2d(in_shape, axes, w2d, _DT[in_dtype], _DT[gy.dtype], pad, pad_value)
    dev = gy.device
    gx = torch.empty(in_shape, dtype=in_dtype, device=dev) if need_dx else None
    gw = torch.empty_like(w2d) if need_dw else None
    ws_bytes = fcfs_backward_workspace(d) if need_dw else 0
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=dev)
    fcfs_backward(d, x.data_ptr() if (x is not None and need_dw) else None, gy.data_ptr(),
                  gx.data_ptr() if gx is not None else None, [gw.data_ptr() if gw is not None else None, None],
                  ws.data_ptr(), ws_bytes, _stream(dev))
    return gx, gw


class FCFSFull2dFunction(torch.autograd.Function):
    """Differentiable non-separable 2D FCFS: forward and both gradients in libfcfs kernels."""

    @staticmethod
    def forward(ctx, x, spec, w2d):
        y = resize_full2d(x, spec["axes"], w2d, spec["pad"], spec["pad_value"], spec.get("out_dtype"))
        ctx.spec = spec
        ctx.save_for_backward(x, w2d)
        return y

    @staticmethod
    def backward(ctx, gy):
        x, w2d = ctx.saved_tensors
        spec = ctx.spec
        need_w = ctx.needs_input_grad[2]
        gx, gw = resize_full2d_backward(x, gy.to(spec.get("out_dtype") or x.dtype), spec["axes"], w2d, spec["pad"],
                                        spec["pad_value"], in_shape=tuple(x.shape), in_dtype=x.dtype,
                                        need_dx=ctx.needs_input_grad[0], need_dw=need_w)
        return gx, None, gw


class FCFSFull2d(torch.nn.Module):
    """FCFS layer with learnable non-separable kernels: weight [C, r_y, r_x, T_y, T_x]
    (or one shared [r_y, r_x, T_y, T_x]) initialised to the outer product of the
    method's two axis tables, from which training may move to any 2D shape."""

    def __init__(self, channels: int, ratios, method: int = BILINEAR, pad: int = PAD_REPLICATE,
                 pad_value: float = 0.0, K: int = 0, per_channel: bool = True, out_dtype=None):
        super().__init__()
        (ry, sy), (rx, sx) = [tuple(rs) for rs in ratios]
        wy, ky = fcfs_make_weights(method, ry, sy, K)
        wx, kx = fcfs_make_weights(method, rx, sx, K)
        w = np.einsum("am,bn->abmn", wy, wx).astype(np.float32)
        if per_channel:
            w = np.tile(w[None], (channels, 1, 1, 1, 1))
        self.weight = torch.nn.Parameter(torch.from_numpy(np.ascontiguousarray(w)))
        self.axes = [Axis(ry, sy, method, ky), Axis(rx, sx, method, kx)]
        self.pad, self.pad_value, self.out_dtype = pad, pad_value, out_dtype

    def forward(self, x):
        spec = {"axes": self.axes, "pad": self.pad, "pad_value": self.pad_value, "out_dtype": self.out_dtype}
        return FCFSFull2dFunction.apply(x, spec, self.weight.contiguous())


# ----------------------------------------------------------------- serving

class _DeviceArray:
    """Minimal __cuda_array_interface__ view of library-owned device memory."""

    def __init__(self, ptr: int, shape, dtype: torch.dtype):
        typestr = {torch.float32: "<f4", torch.bfloat16: "<i2", torch.uint8: "|u1"}[dtype]
        self.__cuda_array_interface__ = {"data": (ptr, False), "shape": tuple(shape), "typestr": typestr,
                                         "version": 3, "strides": None}


class Server:
    """Continuous-batching FCFS server (fcfs_serve_* of libfcfs).

    Requests are 2D images x [1, C, H, W] (uint8, float32 or bfloat16 CUDA
    tensors, kept alive by the server until they complete) resized by one
    (r, s) factor and fixed method on both axes."""

    def __init__(self, hbm_budget_bytes: int, max_inflight: int = 64, out_dtype=torch.float32,
                 tile_budget_per_step: int = 4096, timeout_ms: int = 60_000, auto_release: bool = True,
                 stream: Optional[torch.cuda.Stream] = None):
        self._lib = N.load()
        cfg = N.fcfs_serve_config()
        cfg.hbm_budget_bytes = int(hbm_budget_bytes)
        cfg.max_inflight = int(max_inflight)
        cfg.out_dtype = _DT[out_dtype]
        cfg.tile_budget_per_step = int(tile_budget_per_step)
        cfg.timeout_ms = int(timeout_ms)
        cfg.auto_release = 1 if auto_release else 0
        self.out_dtype = out_dtype
        self._h = ctypes.c_void_p()
        check(self._lib.fcfs_serve_create(ctypes.byref(cfg), stream.cuda_stream if stream is not None else None,
                                          ctypes.byref(self._h)), "fcfs_serve_create")
        self._keep = {}
        self._shapes = {}

    @staticmethod
    def clock() -> float:
        return N.load().fcfs_serve_clock()

    def submit(self, x: torch.Tensor, ratio, method: int = BILINEAR, y: Optional[torch.Tensor] = None,
               arrival: Optional[float] = None, pad: int = PAD_REPLICATE, pad_value: float = 0.0,
               align: int = ALIGN_PAPER, cubic_a: float = 0.0, antialias: bool = False) -> int:
        r, s = ratio
        axes = [Axis(r, s, method)] * 2
        dout = _DT[y.dtype] if y is not None else _DT[self.out_dtype]
        d = make_desc(x.shape, axes, _DT[x.dtype], dout, pad, pad_value, align, cubic_a, antialias)
        rid = ctypes.c_ulonglong()
        t = self.clock() if arrival is None else float(arrival)
        check(self._lib.fcfs_serve_submit(self._h, ctypes.byref(d), x.data_ptr(),
                                          y.data_ptr() if y is not None else None, t, ctypes.byref(rid)),
              "fcfs_serve_submit")
        self._keep[rid.value] = (x, y)
        self._shapes[rid.value] = out_shape(x.shape, axes)
        return rid.value

    def submit_raw(self, desc: N.fcfs_desc, x_ptr: int, y_ptr: Optional[int], arrival: float) -> int:
        """fcfs_serve_submit with a prebuilt descriptor (the caller keeps x alive)."""
        rid = ctypes.c_ulonglong()
        check(self._lib.fcfs_serve_submit(self._h, ctypes.byref(desc), x_ptr, y_ptr, float(arrival),
                                          ctypes.byref(rid)), "fcfs_serve_submit")
        return rid.value

    def submit_batch_raw(self, descs, x_ptrs, y_ptrs, arrivals) -> list:
        """fcfs_serve_submit_batch with prebuilt descriptors (the caller keeps the inputs alive);
        y_ptrs may be None (every output pooled).  Returns the ids; raises on the first invalid
        request (the ones before it stay queued)."""
        n = len(descs)
        if n == 0:
            return []
        darr = (N.fcfs_desc * n)(*descs)
        xarr = (ctypes.c_void_p * n)(*x_ptrs)
        yarr = (ctypes.c_void_p * n)(*y_ptrs) if y_ptrs is not None else None
        tarr = (ctypes.c_double * n)(*[float(t) for t in arrivals])
        ids = (ctypes.c_ulonglong * n)()
        done = ctypes.c_int()
        check(self._lib.fcfs_serve_submit_batch(self._h, n, darr, xarr, yarr, tarr, ids, ctypes.byref(done)),
              "fcfs_serve_submit_batch")
        return list(ids)

    def poll(self, max_ids: int = 4096):
        ids = (ctypes.c_ulonglong * max_ids)()
        n = ctypes.c_int()
        check(self._lib.fcfs_serve_poll(self._h, ids, max_ids, ctypes.byref(n)), "fcfs_serve_poll")
        out = [ids[k] for k in range(n.value)]
        for rid in out:
            self._keep.pop(rid, None)
        return out

    def result(self, rid: int) -> torch.Tensor:
        """Zero-copy view of a pooled output (servers created with auto_release=False)."""
        p = ctypes.c_void_p()
        check(self._lib.fcfs_serve_result(self._h, rid, ctypes.byref(p)), "fcfs_serve_result")
        view = torch.as_tensor(_DeviceArray(p.value, self._shapes[rid], self.out_dtype), device="cuda")
        return view.view(torch.bfloat16) if self.out_dtype == torch.bfloat16 else view

    def release(self, rid: int) -> None:
        check(self._lib.fcfs_serve_release(self._h, rid), "fcfs_serve_release")

    def cancel(self, rid: int) -> None:
        """Give up on a request: queued ones leave at once, running ones stop receiving tiles."""
        check(self._lib.fcfs_serve_cancel(self._h, rid), "fcfs_serve_cancel")

    def drain(self, timeout_ms: int = -1) -> None:
        check(self._lib.fcfs_serve_drain(self._h, timeout_ms), "fcfs_serve_drain")

    def stats(self) -> dict:
        st = N.fcfs_serve_stats_t()
        check(self._lib.fcfs_serve_stats(self._h, ctypes.byref(st)), "fcfs_serve_stats")
        return {name: getattr(st, name) for name, _ in st._fields_}

    def close(self) -> None:
        if self._h:
            check(self._lib.fcfs_serve_destroy(self._h), "fcfs_serve_destroy")
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
