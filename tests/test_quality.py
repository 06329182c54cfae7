"""CPU pins of the image-quality measures (paper_2203_10670_gb300.quality):
PSNR from its closed form, SSIM against a brute-force evaluation of the index
written out window by window from its definition (Wang et al. 2004), and
their basic properties."""
import math

import numpy as np
import pytest
import torch

from paper_2203_10670_gb300 import quality


def _ssim_bruteforce(x, y, L, win=11, sigma=1.5):
    # every window position where the 11 x 11 window fits, one at a time, in float64
    t = np.arange(win) - (win - 1) / 2.0
    g1 = np.exp(-t * t / (2 * sigma * sigma))
    g1 /= g1.sum()
    w = np.outer(g1, g1)
    c1, c2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    vals = []
    H, W = x.shape
    for i in range(H - win + 1):
        for j in range(W - win + 1):
            px, py = x[i:i + win, j:j + win], y[i:i + win, j:j + win]
            mx, my = (w * px).sum(), (w * py).sum()
            vx = (w * (px - mx) ** 2).sum()
            vy = (w * (py - my) ** 2).sum()
            cxy = (w * (px - mx) * (py - my)).sum()
            vals.append(((2 * mx * my + c1) * (2 * cxy + c2)) / ((mx * mx + my * my + c1) * (vx + vy + c2)))
    return float(np.mean(vals))


def test_psnr_closed_form():
    a = torch.zeros(1, 1, 8, 8, dtype=torch.float64)
    b = torch.full((1, 1, 8, 8), 0.1, dtype=torch.float64)
    assert abs(quality.psnr(a, b) - 20.0) < 1e-12  # 10 log10(1 / 0.01)
    assert abs(quality.psnr(a, 2 * b, data_range=255.0) - 10 * math.log10(255.0 ** 2 / 0.04)) < 1e-12
    assert quality.psnr(b, b) == math.inf


@pytest.mark.parametrize("seed", (0, 1, 2))
def test_ssim_matches_windowed_definition(seed):
    rng = np.random.default_rng(seed)
    x = rng.random((19, 23))
    y = np.clip(x + 0.1 * rng.standard_normal(x.shape), 0, 1)
    want = _ssim_bruteforce(x, y, 1.0)
    got = quality.ssim(torch.from_numpy(x)[None, None], torch.from_numpy(y)[None, None])
    assert abs(got - want) < 1e-12
    # channels and images are averaged
    xs = torch.from_numpy(np.stack([x, y]))[None]
    ys = torch.from_numpy(np.stack([y, x]))[None]
    assert abs(quality.ssim(xs, ys) - want) < 1e-12


def test_ssim_properties():
    rng = np.random.default_rng(5)
    x = torch.from_numpy(rng.random((2, 3, 30, 40)))
    y = torch.from_numpy(rng.random((2, 3, 30, 40)))
    assert abs(quality.ssim(x, x) - 1.0) < 1e-12
    assert abs(quality.ssim(x, y) - quality.ssim(y, x)) < 1e-12
    assert quality.ssim(x, y) < 0.2  # unrelated noise images
    with pytest.raises(ValueError):
        quality.ssim(x[:, :, :5], y[:, :, :5])
