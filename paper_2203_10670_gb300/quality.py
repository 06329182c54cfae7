"""Image-quality measures for comparing resize results (the paper's second
experiment compares FCFS with the framework's resize by PSNR and SSIM).

These are evaluation helpers on torch tensors, not part of the FCFS layer:
  psnr(a, b, data_range)  10 log10(data_range^2 / mean((a - b)^2)), in dB;
  ssim(a, b, data_range)  the structural similarity index of Wang, Bovik,
                          Sheikh and Simoncelli (2004): local means, variances
                          and covariance under an 11 x 11 Gaussian window
                          (sigma 1.5), constants (0.01 L)^2 and (0.03 L)^2,
                          averaged over every position where the window fits
                          inside the image, per channel, then over channels
                          and images.
Inputs are [n, c, H, W] tensors of the same shape; arithmetic in float64.
"""
from __future__ import annotations

import math

import torch
import torch.nn.functional as TF


def psnr(a: torch.Tensor, b: torch.Tensor, data_range: float = 1.0) -> float:
    mse = float(((a.double() - b.double()) ** 2).mean())
    return math.inf if mse == 0.0 else 10.0 * math.log10(data_range * data_range / mse)


def _gauss(size: int, sigma: float, device) -> torch.Tensor:
    t = torch.arange(size, dtype=torch.float64, device=device) - (size - 1) / 2.0
    g = torch.exp(-t * t / (2.0 * sigma * sigma))
    return g / g.sum()


def ssim(a: torch.Tensor, b: torch.Tensor, data_range: float = 1.0, window: int = 11, sigma: float = 1.5) -> float:
    if a.shape != b.shape or a.dim() != 4:
        raise ValueError("ssim takes two [n, c, H, W] tensors of the same shape")
    n, c, H, W = a.shape
    if H < window or W < window:
        raise ValueError(f"images smaller than the {window} x {window} window")
    x = a.double().reshape(n * c, 1, H, W)
    y = b.double().reshape(n * c, 1, H, W)
    g = _gauss(window, sigma, x.device)
    kx = g.view(1, 1, 1, window)
    ky = g.view(1, 1, window, 1)

    def blur(t):  # separable Gaussian, valid positions only
        return TF.conv2d(TF.conv2d(t, kx), ky)

    mx, my = blur(x), blur(y)
    sxx = blur(x * x) - mx * mx
    syy = blur(y * y) - my * my
    sxy = blur(x * y) - mx * my
    c1 = (0.01 * data_range) ** 2
    c2 = (0.03 * data_range) ** 2
    s = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
    return float(s.mean())
