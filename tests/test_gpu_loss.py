"""The image loss of Sec. 3.6 on the GPU (ts_image_loss) against the FP64
oracle (oracle/loss.py): 0.8 L1 + 0.2 (1 - SSIM) and its gradient."""
import numpy as np
import pytest
import torch

from oracle import loss as OL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2506_13348_b300 as P
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return P


def gpu_loss(P, x, y, lam=0.2):
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    yd = torch.from_numpy(y.astype(np.float32)).cuda()
    loss = torch.zeros(1, device="cuda")
    grad = torch.full_like(xd, 7.0)
    P.image_loss(xd, yd, loss, grad, lam)
    torch.cuda.synchronize()
    return float(loss.item()), grad.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("shape", [(29, 37), (64, 64), (96, 130), (800, 800)])
def test_image_loss_matches_oracle(P, shape):
    H, W = shape
    rng = np.random.default_rng(H * 1000 + W)
    y = rng.uniform(size=(H, W, 4))
    # a rendered-looking image: the target plus smooth and noisy deviations
    yy, xx = np.mgrid[0:H, 0:W]
    x = np.clip(y + 0.1 * np.sin(xx / 7.0)[..., None] + rng.normal(0, 0.05, size=y.shape), 0, 1)
    ref_loss, ref_grad, _, _ = OL.image_loss(x.astype(np.float32).astype(np.float64),
                                             y.astype(np.float32).astype(np.float64))
    loss, grad = gpu_loss(P, x, y)
    assert abs(loss - ref_loss) <= 2e-6 * max(1.0, abs(ref_loss)), (loss, ref_loss)
    gmax = np.abs(ref_grad).max()
    err = np.abs(grad - ref_grad).max()
    assert err <= 1e-3 * gmax, (err, gmax)
    assert np.all(grad[..., 3] == 0.0)


def test_identical_images_and_pure_l1(P):
    rng = np.random.default_rng(5)
    x = rng.uniform(size=(50, 70, 4))
    loss, grad = gpu_loss(P, x, x)
    assert abs(loss) <= 1e-6
    assert np.abs(grad).max() <= 1e-9
    y = rng.uniform(size=x.shape)
    loss0, grad0 = gpu_loss(P, x, y, lam=0.0)
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    yd = torch.from_numpy(y.astype(np.float32)).cuda()
    l1 = torch.zeros(1, device="cuda")
    g1 = torch.empty_like(xd)
    P.l1_loss(xd, yd, l1, g1)
    torch.cuda.synchronize()
    assert abs(loss0 - float(l1.item())) <= 1e-6
    np.testing.assert_allclose(grad0, g1.cpu().numpy(), rtol=1e-6, atol=1e-12)


def test_bad_arguments(P):
    from paper_2506_13348_b300._lib import TexSplatError
    x = torch.zeros(8, 8, 4, device="cuda")
    loss = torch.zeros(1, device="cuda")
    with pytest.raises(TexSplatError, match="TS_ERR_ARG"):
        P.image_loss(x, x, loss, x.clone(), 1.5)
