"""Optimiser step and multi-view training step."""
import numpy as np
import pytest
import torch

import scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2506_13348_b300 as P
    return P


@pytest.mark.parametrize("n,shadow", [(1 << 20, "bf16"), (1000003, "f16"), (4099, "f32"), (7, None)])
def test_adam_matches_reference_formula(P, n, shadow):
    g = torch.Generator(device="cpu").manual_seed(n)
    p = torch.randn(n, generator=g).cuda()
    gr = torch.randn(n, generator=g).cuda()
    m = torch.randn(n, generator=g).cuda() * 0.1
    v = torch.rand(n, generator=g).cuda() * 0.1
    p0, g0, m0, v0 = p.double(), gr.double(), m.double(), v.double()
    lr, b1, b2, eps, step = 1e-2, 0.9, 0.999, 1e-8, 7
    sh = {"bf16": torch.bfloat16, "f16": torch.float16, "f32": torch.float32}
    out = torch.empty(n, dtype=sh[shadow], device="cuda") if shadow else None
    P.adam_update(p, gr, m, v, step, lr, b1, b2, eps, shadow_ptr=out.data_ptr() if shadow else 0,
                  shadow_dtype=shadow or "f32", zero_grad=True)
    torch.cuda.synchronize()
    m1 = b1 * m0 + (1 - b1) * g0
    v1 = b2 * v0 + (1 - b2) * g0 * g0
    p1 = p0 - lr * (m1 / (1 - b1 ** step)) / ((v1 / (1 - b2 ** step)).sqrt() + eps)
    np.testing.assert_allclose(m.double().cpu(), m1.cpu(), rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(v.double().cpu(), v1.cpu(), rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(p.double().cpu(), p1.cpu(), rtol=1e-5, atol=1e-6)
    assert torch.count_nonzero(gr).item() == 0
    if shadow:
        assert torch.equal(out, p.to(sh[shadow]))  # round to nearest even of the master


def test_training_steps_reduce_loss(P):
    scene = sg.make_scene(1, n=4000, T=8, seed=40)
    env = sg.make_env(4, cube_res=16, irr_res=8, lut_res=32)
    sc = P.Scene.from_arrays(scene, env, store="bf16")
    cams = [sg.look_at_camera(e, 96, 96) for e in [(3.0, 0.5, 0.5), (0.5, 3.0, 0.2), (-2.0, -2.0, 1.0),
                                                   (0.3, -0.4, 3.2)]]
    # targets: the renders of a perturbed-texture copy of the scene
    tgt_scene = dict(scene, texels=np.clip(scene["texels"] * 0.5 + 0.25, 0, 1).astype(np.float32))
    tsc = P.Scene.from_arrays(tgt_scene, env)
    targets = [P.render(tsc, c)[0].clone() for c in cams]
    tr = P.Trainer(sc, scene, store="bf16", lr_tex=2e-2)
    losses = [tr.step(cams, targets).sum().item() for _ in range(30)]
    assert np.isfinite(losses).all()
    assert losses[-1] < 0.8 * losses[0], losses


def test_training_with_the_paper_objective(P):
    """0.8 L1 + 0.2 D-SSIM + 0.05 L_n (Sec. 3.6): finite and decreasing."""
    scene = sg.make_scene(1, n=4000, T=8, seed=41)
    env = sg.make_env(4, cube_res=16, irr_res=8, lut_res=32)
    sc = P.Scene.from_arrays(scene, env, store="bf16")
    cams = [sg.look_at_camera(e, 96, 96) for e in [(3.0, 0.5, 0.5), (0.5, 3.0, 0.2), (-2.0, -2.0, 1.0)]]
    tgt_scene = dict(scene, texels=np.clip(scene["texels"] * 0.5 + 0.25, 0, 1).astype(np.float32))
    tsc = P.Scene.from_arrays(tgt_scene, env)
    targets = [P.render(tsc, c)[0].clone() for c in cams]
    tr = P.Trainer(sc, scene, store="bf16", lr_tex=2e-2, lambda_dssim=0.2, normal_weight=0.05)
    losses = [tr.step(cams, targets).sum().item() for _ in range(30)]
    assert np.isfinite(losses).all()
    assert losses[-1] < 0.9 * losses[0], losses


def test_training_the_environment_and_indirect_light(P):
    """lr_env / lr_sh: the stored cubes and SH follow the Adam masters (a
    fresh scene built from the masters renders the same image) and learning
    the environment alone pulls the render towards a target lit by a
    brighter environment."""
    scene = sg.make_scene(1, n=3000, T=4, seed=42)
    rng = np.random.default_rng(3)
    scene["sh"] = (rng.normal(size=(3000, 4, 3)) * 0.2).astype(np.float32)
    env = sg.make_env(5, cube_res=16, levels=2, irr_res=8, lut_res=32)
    bright = dict(env, spec=[np.clip(m * 1.6 + 0.05, 0, None).astype(np.float32) for m in env["spec"]],
                  irr=(env["irr"] * 1.6 + 0.05).astype(np.float32))
    cams = [sg.look_at_camera(e, 96, 96) for e in [(3.0, 0.5, 0.5), (0.5, 3.0, 0.2), (-2.0, -2.0, 1.0)]]
    vis = torch.full((96, 96), 0.7, device="cuda")
    cams = [dict(c, vis=vis) for c in cams]
    tsc = P.Scene.from_arrays(scene, bright)
    targets = [P.render(tsc, c)[0].clone() for c in cams]
    sc = P.Scene.from_arrays(scene, env, store="f32")
    tr = P.Trainer(sc, scene, store="f32", lr_geom=0.0, lr_tex=0.0, env=env, lr_env=1e-2, lr_sh=1e-2)
    losses = [tr.step(cams, targets).sum().item() for _ in range(25)]
    assert np.isfinite(losses).all()
    assert losses[-1] < 0.7 * losses[0], losses
    # the SH and cubes moved, and the stored copies are the masters
    assert not np.allclose(tr.master["sh"].cpu().numpy(), scene["sh"])
    spec_sizes = [m.size for m in env["spec"]]
    flat = tr.master["spec"].cpu().numpy()
    parts = np.split(flat, np.cumsum(spec_sizes)[:-1])
    env2 = dict(env, spec=[p.reshape(m.shape) for p, m in zip(parts, env["spec"])],
                irr=tr.master["irr"].cpu().numpy().reshape(env["irr"].shape))
    assert np.abs(env2["spec"][0] - env["spec"][0]).max() > 1e-3
    geo = {k: tr.master[k].cpu().numpy() for k in ("means", "quats", "scales", "opacity", "texels")}
    ref = P.Scene.from_arrays(dict(scene, **geo, sh=tr.master["sh"].cpu().numpy()), env2, store="f32")
    a, _ = P.render(sc, cams[0])
    b, _ = P.render(ref, cams[0])
    torch.cuda.synchronize()
    assert torch.equal(a, b)
