"""Image reconstruction loss of the training objective (TEST INFRASTRUCTURE).

Sec. 3.6 trains with L_img = (1 - lambda) L_1 + lambda L_D-SSIM, lambda = 0.2.
The paper does not restate SSIM; this module writes out the standard
structural-similarity index of Wang et al. (2004) as the 3DGS line of work
evaluates it (reading R17):

  per RGB channel, with G the normalised 11 x 11 Gaussian window (sigma 1.5)
  applied as a 2-D convolution with zero padding ("same" size):
    mu_x = G * x,  mu_y = G * y,
    s_xx = G * (x x) - mu_x^2,  s_yy = G * (y y) - mu_y^2,  s_xy = G * (x y) - mu_x mu_y,
    SSIM = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2)),
  C1 = 0.01^2, C2 = 0.03^2 (data range 1);
  SSIM = mean over pixels and channels;  L_D-SSIM = 1 - SSIM;
  L_1 = mean over pixels and channels of |x - y|.

Everything is float64 numpy/torch; the convolution is torch's conv2d (a
library primitive), the gradient is autograd of the same expression.

Parity: pinned by tests/test_oracle_loss.py against a direct per-pixel
window sum on tiny images, the closed form on constant images, SSIM(x, x) = 1
and central differences.
"""
from __future__ import annotations

import numpy as np
import torch

F64 = torch.float64
WIN = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2
LAMBDA_DSSIM = 0.2


def gaussian_window(size: int = WIN, sigma: float = SIGMA) -> np.ndarray:
    """Normalised 2-D Gaussian window (outer product of the 1-D one)."""
    r = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-(r * r) / (2.0 * sigma * sigma))
    g /= g.sum()
    return np.outer(g, g)


def _blur(img: torch.Tensor) -> torch.Tensor:
    """[C, H, W] -> G * img per channel, zero padding, same size."""
    w = torch.from_numpy(gaussian_window()).to(F64)[None, None].expand(img.shape[0], 1, WIN, WIN)
    return torch.nn.functional.conv2d(img[None], w, padding=WIN // 2, groups=img.shape[0])[0]


def ssim_map(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """Per-pixel, per-channel SSIM of [C, H, W] images."""
    mx, my = _blur(x), _blur(y)
    sxx = _blur(x * x) - mx * mx
    syy = _blur(y * y) - my * my
    sxy = _blur(x * y) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def image_loss(rgba: np.ndarray, target: np.ndarray, lam: float = LAMBDA_DSSIM):
    """L_img of [H, W, 4] images (RGB used).  Returns (loss, dL/drgba [H, W, 4]
    with a zero alpha column, L_1, SSIM)."""
    x = torch.tensor(np.asarray(rgba, dtype=np.float64)[..., :3]).permute(2, 0, 1).contiguous().requires_grad_(True)
    y = torch.tensor(np.asarray(target, dtype=np.float64)[..., :3]).permute(2, 0, 1).contiguous()
    l1 = (x - y).abs().mean()
    ssim = ssim_map(x, y).mean()
    loss = (1.0 - lam) * l1 + lam * (1.0 - ssim)
    (g,) = torch.autograd.grad(loss, x)
    grad = np.zeros(np.asarray(rgba).shape, dtype=np.float64)
    grad[..., :3] = g.permute(1, 2, 0).numpy()
    return float(loss.detach()), grad, float(l1.detach()), float(ssim.detach())


def ssim_direct(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """SSIM map of [H, W] single-channel images by explicit window sums at
    every pixel (window taps outside the image count as zero).  Slow; for
    tiny images only."""
    H, W = x.shape
    g = gaussian_window()
    h = WIN // 2
    out = np.empty((H, W))
    for i in range(H):
        for j in range(W):
            m = [0.0] * 5
            for a in range(WIN):
                for b in range(WIN):
                    ii, jj = i + a - h, j + b - h
                    if 0 <= ii < H and 0 <= jj < W:
                        w = g[a, b]
                        xv, yv = x[ii, jj], y[ii, jj]
                        m[0] += w * xv
                        m[1] += w * yv
                        m[2] += w * xv * xv
                        m[3] += w * yv * yv
                        m[4] += w * xv * yv
            mx, my = m[0], m[1]
            sxx, syy, sxy = m[2] - mx * mx, m[3] - my * my, m[4] - mx * my
            out[i, j] = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    return out


def ssim_constant_interior(a: float, b: float) -> float:
    """SSIM of two constant images a, b away from the border (window fully
    inside): the variances and covariance vanish."""
    return (2 * a * b + C1) * C2 / ((a * a + b * b + C1) * C2)


__all__ = ["gaussian_window", "ssim_map", "image_loss", "ssim_direct", "ssim_constant_interior",
           "WIN", "SIGMA", "C1", "C2", "LAMBDA_DSSIM"]
