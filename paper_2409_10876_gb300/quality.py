"""Image-quality figures for recovered initial-pressure images (Sec. 4 reports
PSNR and SSIM of the stitched image against the ground truth).

Host-side evaluation only (NumPy): the images come from the GPU path
(deconvolved patches stitched by pact_stitch); nothing here is on the
per-iteration hot path.
"""
from __future__ import annotations

import numpy as np
import torch

from . import pact


def psnr(img: np.ndarray, ref: np.ndarray, data_range: float = 1.0, mask: np.ndarray = None) -> float:
    """10 log10(range^2 / MSE) over the pixels of `mask` (all if None)."""
    d = np.asarray(img, np.float64) - np.asarray(ref, np.float64)
    if mask is not None:
        d = d[mask]
    mse = float(np.mean(d * d))
    return float("inf") if mse == 0.0 else 10.0 * np.log10(data_range ** 2 / mse)


def _gauss_filter(x: np.ndarray, sigma: float = 1.5, radius: int = 5) -> np.ndarray:
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    k /= k.sum()
    y = np.apply_along_axis(lambda r: np.convolve(r, k, mode="same"), 0, x)
    return np.apply_along_axis(lambda r: np.convolve(r, k, mode="same"), 1, y)


def ssim(img: np.ndarray, ref: np.ndarray, data_range: float = 1.0, mask: np.ndarray = None) -> float:
    """Structural similarity with an 11-tap Gaussian window (sigma 1.5),
    K1 = 0.01, K2 = 0.03, averaged over the pixels of `mask` (all if None)."""
    x, y = np.asarray(img, np.float64), np.asarray(ref, np.float64)
    c1, c2 = (0.01 * data_range) ** 2, (0.03 * data_range) ** 2
    mx, my = _gauss_filter(x), _gauss_filter(y)
    sxx = _gauss_filter(x * x) - mx * mx
    syy = _gauss_filter(y * y) - my * my
    sxy = _gauss_filter(x * y) - mx * my
    s = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
    return float(np.mean(s if mask is None else s[mask]))


def recovered_image(pb: "pact.Problem", Y: torch.Tensor, d, eps: float, sos: torch.Tensor) -> np.ndarray:
    """Stitched initial-pressure image (Sec. S1.5) from the deconvolved patches
    X_hat (Eq. 6) at the SOS `sos`."""
    w = pact.sos_to_delays(pb, sos.contiguous())
    Xh = pact.mc_deconv_loss(pb, w, Y, d, eps, want_grad=False, want_xhat=True)["Xhat"]
    return pact.stitch(pb, Xh).cpu().numpy()


def image_mask(cfg) -> np.ndarray:
    """Pixels inside the SOS mask disk (the region the patches cover)."""
    cx = (np.arange(cfg.img_w) - (cfg.img_w - 1) / 2.0) * cfg.dx
    cy = (np.arange(cfg.img_h) - (cfg.img_h - 1) / 2.0) * cfg.dx
    yy, xx = np.meshgrid(cy, cx, indexing="ij")
    return xx * xx + yy * yy <= cfg.mask_radius ** 2
