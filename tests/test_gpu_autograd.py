"""The autograd wrapper on raw optimisation variables (log scales, logit
opacities, unnormalised quaternions) against the oracle with the chain rule
of the activations written out."""
import numpy as np
import pytest
import torch

import scenegen as sg
from oracle import grad as G
from oracle import keys as K
from oracle import render as R
from tests.helpers import check_admissible

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2506_13348_b300 as P
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return P


def test_activation_kernels(P):
    g = torch.Generator().manual_seed(1)
    ls = (torch.randn(1001, 2, generator=g) * 2).cuda()
    lo = (torch.randn(1001, generator=g) * 4).cuda()
    s, o = P.activate(ls, lo)
    torch.cuda.synchronize()
    np.testing.assert_allclose(s.cpu().double(), ls.cpu().double().exp(), rtol=1e-6)
    np.testing.assert_allclose(o.cpu().double(), torch.sigmoid(lo.cpu().double()), rtol=1e-6, atol=1e-7)
    gs, go = torch.randn(1001, 2, generator=g).cuda(), torch.randn(1001, generator=g).cuda()
    gls, glo = P.activate_backward(s, o, gs, go)
    torch.cuda.synchronize()
    np.testing.assert_allclose(gls.cpu(), (gs * s).cpu(), rtol=1e-6)
    np.testing.assert_allclose(glo.cpu(), (go * o * (1 - o)).cpu(), rtol=1e-6, atol=1e-7)


def test_autograd_wrapper_matches_oracle_with_chain_rule(P):
    scene = sg.make_scene(0, n=800, T=4, seed=17)
    env = sg.make_env(2, cube_res=16, levels=2, irr_res=8, lut_res=32)
    cam = sg.look_at_camera((3.0, 0.8, 0.6), 96, 80)
    rng = np.random.default_rng(2)
    # raw variables; the scene the oracle sees is their float32 activation
    log_s = np.log(scene["scales"]).astype(np.float32)
    logit_o = np.log(scene["opacity"] / (1 - scene["opacity"])).astype(np.float32)
    quats_raw = (scene["quats"] * rng.uniform(0.5, 2.0, size=(800, 1))).astype(np.float32)
    dev = torch.device("cuda")
    t = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device=dev, requires_grad=True)  # noqa: E731
    means, quats, ls, lo = t(scene["means"]), t(quats_raw), t(log_s), t(logit_o)
    tex, spec, irr = t(scene["texels"]), t(np.concatenate([m.ravel() for m in env["spec"]])), t(env["irr"])
    lut = torch.tensor(env["lut"], device=dev)
    sc = P.Scene(0)
    sc.levels = len(env["spec"])
    out = P.TexSplatRender.apply(sc, cam, lut, means, quats, ls, lo, tex, spec, irr)
    s_act, o_act = P.activate(ls.detach(), lo.detach())
    torch.cuda.synchronize()
    act_scene = dict(scene, quats=quats_raw, scales=s_act.cpu().numpy(), opacity=o_act.cpu().numpy())
    kl = K.build_keys(act_scene, cam)
    ref = R.render(act_scene, cam, env, keylist=kl)
    check_admissible(out.detach().cpu().numpy(), ref, 1e-4, 1e-3, "autograd wrapper")
    gamb = ref["grad_ambiguous"].numpy()
    dL = rng.normal(size=(80, 96, 4))
    dL[gamb] = 0.0
    (out * torch.tensor(dL, dtype=torch.float32, device=dev)).sum().backward()
    rg = G.render_grads(act_scene, cam, env, dL, keylist=kl)
    s64, o64 = act_scene["scales"].astype(np.float64), act_scene["opacity"].astype(np.float64)
    expect = {"means": rg["means"], "quats": rg["quats"], "texels": rg["texels"],
              "log_scales": rg["scales"] * s64, "logit_opacity": rg["opacity"] * o64 * (1 - o64),
              "irr": rg["irr"]}
    got = {"means": means.grad, "quats": quats.grad, "texels": tex.grad, "log_scales": ls.grad,
           "logit_opacity": lo.grad, "irr": irr.grad}
    for name, r in expect.items():
        g = got[name].cpu().numpy().astype(np.float64).reshape(r.shape)
        scale = np.abs(r).max()
        assert scale > 0, name
        bad = np.abs(g - r) > 1e-3 * scale + 1e-6
        assert not bad.any(), (name, int(bad.sum()), float(np.abs(g - r).max()), float(scale))
