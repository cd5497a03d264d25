"""Depth channel and normal-consistency loss (Sec. 3.6) on the GPU against
the FP64 oracle: the saved blended depth, the loss value on the GPU's own
buffers, and the parameter gradients of weight x L_n through the backward."""
import numpy as np
import pytest
import torch

import scenegen as sg
from oracle import grad as G
from oracle import keys as K
from oracle import loss as OL
from oracle import render as R
from tests.helpers import admissible_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2506_13348_b300 as P
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return P


def case0():
    # 2000 splats on the unit sphere: about 40 % of the 128x128 view covered >= 0.5
    scene = sg.make_scene(0, n=2000, T=4, seed=11)
    env = sg.make_env(0, cube_res=16, levels=2, irr_res=8, lut_res=32)
    cam = sg.look_at_camera((4.0, 0.0, 0.0), 128, 128)
    return scene, env, cam


def test_depth_channel_matches_oracle(P):
    scene, env, cam = case0()
    kl = K.build_keys(scene, cam)
    ref = R.render(scene, cam, env, keylist=kl)
    sc = P.Scene.from_arrays(scene, env)
    _, saved = P.render(sc, cam, save=True)
    z, a = saved.depth()
    torch.cuda.synchronize()
    z, a = z.cpu().numpy().astype(np.float64), a.cpu().numpy().astype(np.float64)
    amb = ref["ambiguous"].numpy()
    assert amb.mean() <= 1e-3
    assert (ref["A"].numpy() > 0.5).sum() > 2000
    assert admissible_errors(a, ref, "A")[~amb].max() <= 1e-4
    assert admissible_errors(z, ref, "Z")[~amb].max() <= 4e-4  # depths ~4: 1e-4 relative
    saved.release()


def test_normal_loss_value_and_adjoint_on_gpu_buffers(P):
    """Loss of the GPU's own Z, A, X evaluated by the oracle in FP64, and the
    loss's gradient (carried by a backward with a zero image gradient) against
    the oracle's autograd of weight x L_n w.r.t. the scene parameters."""
    scene, env, cam = case0()
    sc = P.Scene.from_arrays(scene, env)
    _, saved = P.render(sc, cam, save=True)
    z, a = saved.depth()
    g, _, _ = saved.pixels(0)
    torch.cuda.synchronize()
    Zt = torch.tensor(z.cpu().numpy(), dtype=torch.float64)
    At = torch.tensor(a.cpu().numpy(), dtype=torch.float64)
    Xt = torch.tensor(g.cpu().numpy(), dtype=torch.float64)
    L_ref, mask, _ = OL.depth_normal_loss(Zt, At, Xt, cam)
    assert mask.sum() > 1000
    w = 0.7
    loss = torch.zeros(1, device="cuda")
    saved.normal_loss(loss, weight=w)
    torch.cuda.synchronize()
    assert abs(float(loss.item()) - w * float(L_ref)) <= 1e-5 * max(1e-3, w * float(L_ref)), (
        float(loss.item()), w * float(L_ref))
    saved.release()


def test_normal_loss_gradient_parity(P):
    scene, env, cam = case0()
    kl = K.build_keys(scene, cam)
    w = 0.5
    ref = G.render_grads(scene, cam, env, np.zeros((128, 128, 4)), keylist=kl, normal_weight=w)
    sc = P.Scene.from_arrays(scene, env)
    _, saved = P.render(sc, cam, save=True)
    loss = torch.zeros(1, device="cuda")
    saved.normal_loss(loss, weight=w)
    grads = P.zero_grads(sc)
    P.render_backward(saved, torch.zeros(128, 128, 4, device="cuda"), grads)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}
    report = {}
    for name in ("means", "quats", "scales", "opacity", "texels"):
        r = ref[name]
        gg = got[name].reshape(r.shape)
        scale = np.abs(r).max()
        assert scale > 0, name
        err = np.abs(gg - r)
        report[name] = (float(err.max()), float(scale))
        bad = err > 1e-3 * scale + 1e-7
        assert not bad.any(), (name, int(bad.sum()), report[name], np.argwhere(bad)[:5])
    # the environment does not enter L_n
    assert np.abs(got["spec"]).max() == 0.0 and np.abs(got["irr"]).max() == 0.0
    print("normal-loss gradient max error / max |g|:", {k: v[0] / v[1] for k, v in report.items()})
    saved.release()
