"""Image reconstruction loss of the training objective (TEST INFRASTRUCTURE).

Sec. 3.6 trains with L_img = (1 - lambda) L_1 + lambda L_D-SSIM, lambda = 0.2.
The paper does not restate SSIM; this module writes out the standard
structural-similarity index of Wang et al. (2004) as the 3DGS line of work
evaluates it (the paper names D-SSIM and lambda only; window, padding,
constants and the RGB-only mean below are those conventions):

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

Normal consistency (Sec. 3.6 gives only L_n = 1 - N~^T N; the depth kind,
the stencil and the treatment of background below follow 2DGS): the rendered
depth is the expected depth D = Z / A of the blended camera depth Z and the
coverage A; each pixel is back-projected to P = D (x'/fx, y'/fy, 1) in camera
space; the depth normal is N~ = normalize((P[y+1] - P[y-1]) x (P[x+1] - P[x-1]))
(central differences, facing the camera), turned to world space by R^T; N is
the normalised blended normal channel.  A pixel counts when it is interior and
it and its four neighbours have coverage >= 0.5 (a surface is there) and its
normal and cross product are non-zero; L_n = sum over counted pixels of
(1 - N~ . N) / ((W - 2)(H - 2)).

Parity: pinned by tests/test_oracle_loss.py against a direct per-pixel
window sum on tiny images, the closed form on constant images, SSIM(x, x) = 1,
central differences, and for L_n by planes in closed form (tests/test_oracle_render.py).
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


NORMAL_COVER_MIN = 0.5


def depth_normal_loss(Z: torch.Tensor, A: torch.Tensor, X: torch.Tensor, cam: dict):
    """L_n of [H, W] blended depth Z and coverage A and the [H, W, 8] G-buffer
    X (normal channels 5-7), float64 torch (differentiable).  Returns
    (L_n, counted mask [H, W] bool, depth normal in world space [H, W, 3])."""
    H, W = Z.shape
    R = torch.tensor(np.asarray(cam["R"], dtype=np.float64))
    fx, fy, cx, cy = (float(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    xs = (torch.arange(W, dtype=F64) + 0.5 - cx) / fx
    ys = (torch.arange(H, dtype=F64) + 0.5 - cy) / fy
    ok_a = A >= NORMAL_COVER_MIN
    D = torch.where(ok_a, Z / torch.where(ok_a, A, torch.ones_like(A)), torch.zeros_like(Z))
    P = torch.stack([D * xs[None, :], D * ys[:, None], D], -1)  # [H, W, 3] camera space
    dx = P[1:-1, 2:] - P[1:-1, :-2]
    dy = P[2:, 1:-1] - P[:-2, 1:-1]
    c = torch.cross(dy, dx, dim=-1)
    cn = torch.linalg.vector_norm(c, dim=-1)
    N = X[1:-1, 1:-1, 5:8]
    nn = torch.linalg.vector_norm(N, dim=-1)
    valid = ok_a[1:-1, 1:-1] & ok_a[1:-1, 2:] & ok_a[1:-1, :-2] & ok_a[2:, 1:-1] & ok_a[:-2, 1:-1]
    valid = valid & (nn >= 1e-12) & (cn > 0)
    one = torch.ones_like(cn)
    Nt_c = c / torch.where(valid, cn, one)[..., None]
    Nt_w = Nt_c @ R  # R^T n, row-vector form
    Nh = N / torch.where(valid, nn, one)[..., None]
    term = torch.where(valid, 1.0 - (Nt_w * Nh).sum(-1), torch.zeros_like(cn))
    L = term.sum() / float((W - 2) * (H - 2))
    mask = torch.zeros(H, W, dtype=torch.bool)
    mask[1:-1, 1:-1] = valid
    full = torch.zeros(H, W, 3, dtype=F64)
    full[1:-1, 1:-1] = Nt_w.detach()
    return L, mask, full


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
           "depth_normal_loss", "WIN", "SIGMA", "C1", "C2", "LAMBDA_DSSIM", "NORMAL_COVER_MIN"]
