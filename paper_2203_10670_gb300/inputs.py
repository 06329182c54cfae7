"""Seeded synthetic inputs for the FCFS workloads.

Holds none of the method's arithmetic: only shapes, seeds and value
distributions.  Both the CUDA path (tests, bench) and the FP64 oracle are fed
from these tensors, so they see identical bits.

Workloads (spatial axes outermost first):
  c1  one image 1x1x64x64, U[0,1), seed 0, bilinear 3/2 both axes, replicate
  c2  16x3x1080x1920, U[0,1), seed 1: bicubic 2/3, bicubic 4/3, nearest 3/2
  c3  8x64x256x256, N(0,1) rounded to bf16, seed 2; upstream gradient seed 3;
      learnable per-channel taps initialised to bilinear, scale 5/4
  c4  serving: 10,000 requests, C=3 uint8 U{0..255}; H, W log-uniform in
      [64, 2048] (seed 4); r/s uniform over {1/2,2/3,3/4,4/3,3/2,5/2};
      method uniform over nearest/bilinear/bicubic; Poisson arrivals (seed 5)
  c5  1x3x8192x8192 U[0,1) seed 6 (bicubic 7/5); 1x1x256x256x256 U[0,1)
      seed 7 (trilinear 3/2)
  quality comparison (the paper's second experiment): 1x3x1024x1024 images
      with a natural-image (1/f) spectrum, seed 12
"""
from __future__ import annotations

import math

import numpy as np
import torch

C1 = dict(shape=(1, 1, 64, 64), seed=0)
C2 = dict(shape=(16, 3, 1080, 1920), seed=1)
C3 = dict(shape=(8, 64, 256, 256), seed=2, grad_seed=3, ratio=(5, 4))
C4 = dict(count=10_000, channels=3, size_seed=4, arrival_seed=5, hw_range=(64, 2048),
          ratios=((1, 2), (2, 3), (3, 4), (4, 3), (3, 2), (5, 2)))
C5_2D = dict(shape=(1, 3, 8192, 8192), seed=6, ratio=(7, 5))
C5_3D = dict(shape=(1, 1, 256, 256, 256), seed=7, ratio=(3, 2))


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


def uniform(shape, seed: int, device="cpu", dtype=torch.float32) -> torch.Tensor:
    """U[0, 1) drawn in float32 (then cast)."""
    x = torch.rand(shape, generator=_gen(seed, device), device=device, dtype=torch.float32)
    return x if dtype == torch.float32 else x.to(dtype)


def normal(shape, seed: int, device="cpu", dtype=torch.float32) -> torch.Tensor:
    """N(0, 1) drawn in float32; bf16 values are the round-to-nearest of those draws."""
    x = torch.randn(shape, generator=_gen(seed, device), device=device, dtype=torch.float32)
    return x if dtype == torch.float32 else x.to(dtype)


def natural_image(shape, seed: int, device="cpu", dtype=torch.float32) -> torch.Tensor:
    """Images [n, c, H, W] with the 1/f amplitude spectrum of natural photographs
    (random phases from the seed), each plane scaled to [0, 1]: smooth regions and
    edges at every scale, a stand-in for photographs such as face images."""
    n, c, H, W = shape
    g = torch.Generator().manual_seed(seed)
    fy = torch.fft.fftfreq(H, dtype=torch.float64)[:, None]
    fx = torch.fft.rfftfreq(W, dtype=torch.float64)[None, :]
    f = torch.sqrt(fy * fy + fx * fx)
    f[0, 0] = 1.0
    phase = torch.rand((n, c, H, W // 2 + 1), generator=g, dtype=torch.float64) * (2 * math.pi)
    img = torch.fft.irfft2(torch.polar(1.0 / f, phase), s=(H, W))
    lo = img.amin(dim=(2, 3), keepdim=True)
    hi = img.amax(dim=(2, 3), keepdim=True)
    return ((img - lo) / (hi - lo)).to(device=device, dtype=dtype)


def uint8_pixels(shape, seed: int, device="cpu") -> torch.Tensor:
    """Uniform integers 0..255."""
    return torch.randint(0, 256, shape, generator=_gen(seed, device), device=device, dtype=torch.uint8)


def serving_requests(count: int = C4["count"], size_seed: int = C4["size_seed"], arrival_seed: int = C4["arrival_seed"],
                     rate_per_s: float = 1000.0):
    """Request list: dicts with H, W, r, s, method and arrival time (seconds)."""
    rng = np.random.default_rng(size_seed)
    lo, hi = C4["hw_range"]
    H = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), count))).astype(int)
    W = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), count))).astype(int)
    ratio_idx = rng.integers(0, len(C4["ratios"]), count)
    method = rng.integers(0, 3, count)
    arr = np.random.default_rng(arrival_seed)
    gaps = arr.exponential(1.0 / rate_per_s, count)
    t = np.cumsum(gaps)
    out = []
    for k in range(count):
        r, s = C4["ratios"][ratio_idx[k]]
        out.append(dict(H=int(H[k]), W=int(W[k]), r=r, s=s, method=int(method[k]), arrival=float(t[k])))
    return out
