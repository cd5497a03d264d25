"""Pins of the oracle's image loss (oracle/loss.py): L_img = 0.8 L_1 + 0.2 (1 - SSIM)."""
import numpy as np
import torch

from oracle import loss as L


def test_window_is_normalised_gaussian():
    g = L.gaussian_window()
    assert g.shape == (11, 11)
    assert abs(g.sum() - 1.0) < 1e-15
    # separable: rank one, symmetric, peak in the centre, ratio to the
    # neighbouring tap exp(-1/(2 sigma^2))
    assert np.linalg.matrix_rank(g) == 1
    np.testing.assert_allclose(g, g.T, rtol=0, atol=0)
    assert g[5, 5] == g.max()
    np.testing.assert_allclose(g[5, 6] / g[5, 5], np.exp(-1.0 / (2 * 1.5 ** 2)), rtol=1e-14)


def test_ssim_map_equals_direct_window_sums():
    rng = np.random.default_rng(0)
    x = rng.uniform(size=(7, 9))
    y = np.clip(x + rng.normal(0, 0.2, size=x.shape), 0, 1)
    ref = L.ssim_direct(x, y)
    got = L.ssim_map(torch.tensor(x)[None], torch.tensor(y)[None])[0].numpy()
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-14)


def test_ssim_of_identical_images_is_one():
    rng = np.random.default_rng(1)
    img = rng.uniform(size=(20, 24, 4))
    loss, grad, l1, ssim = L.image_loss(img, img)
    assert l1 == 0.0
    assert abs(ssim - 1.0) < 1e-14
    assert abs(loss) < 1e-14
    # SSIM is maximal at y = x, and L1's subgradient is taken as 0 there
    assert np.abs(grad).max() < 1e-12


def test_constant_images_closed_form_in_the_interior():
    a, b = 0.3, 0.7
    x = torch.full((1, 30, 30), a, dtype=torch.float64)
    y = torch.full((1, 30, 30), b, dtype=torch.float64)
    m = L.ssim_map(x, y)[0].numpy()
    np.testing.assert_allclose(m[5:-5, 5:-5], L.ssim_constant_interior(a, b), rtol=1e-12)
    # near the border the zero padding lowers the window mass: not the interior value
    assert abs(m[0, 0] - L.ssim_constant_interior(a, b)) > 1e-3


def test_l1_part_and_weights():
    rng = np.random.default_rng(2)
    x = rng.uniform(size=(12, 16, 4))
    y = rng.uniform(size=(12, 16, 4))
    loss, grad, l1, ssim = L.image_loss(x, y)
    np.testing.assert_allclose(l1, np.abs(x[..., :3] - y[..., :3]).mean(), rtol=1e-14)
    np.testing.assert_allclose(loss, 0.8 * l1 + 0.2 * (1 - ssim), rtol=1e-14)
    assert np.all(grad[..., 3] == 0.0)
    # pure L1 (lambda 0): the gradient is sign / (3 N)
    _, g1, _, _ = L.image_loss(x, y, lam=0.0)
    np.testing.assert_allclose(g1[..., :3], np.sign(x[..., :3] - y[..., :3]) / (3 * 12 * 16), rtol=1e-14)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    x = rng.uniform(0.1, 0.9, size=(9, 11, 4))
    y = rng.uniform(0.1, 0.9, size=(9, 11, 4))
    _, grad, _, _ = L.image_loss(x, y)
    h = 1e-6
    for (i, j, c) in [(0, 0, 0), (4, 5, 1), (8, 10, 2), (2, 7, 0), (6, 1, 2)]:
        xp, xm = x.copy(), x.copy()
        xp[i, j, c] += h
        xm[i, j, c] -= h
        fd = (L.image_loss(xp, y)[0] - L.image_loss(xm, y)[0]) / (2 * h)
        np.testing.assert_allclose(grad[i, j, c], fd, rtol=1e-6, atol=1e-10)
