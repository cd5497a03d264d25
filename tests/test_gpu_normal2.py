"""Two-component tangent normals (Sec. 3.5.1) on the GPU against the FP64
oracle: images (software, hardware-atlas and flat samplers) and gradients,
alone and with the indirect light."""
import numpy as np
import pytest
import torch

import scenegen as sg
from oracle import grad as G
from oracle import keys as K
from oracle import render as R
from tests.helpers import admissible_errors, check_admissible

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2506_13348_b300 as P
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return P


def xy_scene(seed=3, n=600, const=False):
    scene = sg.make_scene(1, n=n, T=4, seed=seed)
    tex = scene["texels"]
    if const:
        tex[:] = tex[:, :1, :1, :]
    tex[..., 7] = 0.0  # not read under the two-component encoding
    scene["texels"] = np.ascontiguousarray(tex)
    scene["normal_encoding"] = "xy"
    return scene


def test_xy_image_matches_oracle(P):
    scene = xy_scene()
    env = sg.make_env(3, cube_res=16, levels=2, irr_res=8, lut_res=32)
    cam = sg.look_at_camera((2.6, 1.2, 0.8), 96, 80)
    kl = K.build_keys(scene, cam)
    ref = R.render(scene, cam, env, keylist=kl)
    sc = P.Scene.from_arrays(scene, env)
    out, saved = P.render(sc, cam, save=True)
    g, _, _ = saved.pixels(0)
    torch.cuda.synchronize()
    check_admissible(out.cpu().numpy(), ref, 1e-4, 1e-3, "two-component normals")
    amb = ref["ambiguous"].numpy()
    # the blended normal channels carry the rebuilt n_z
    gx = g.cpu().numpy().astype(np.float64).reshape(80, 96, 8)
    gerr = admissible_errors(gx, ref, "X")
    assert gerr[~amb].max() <= 1e-4
    # and the encoding matters: the three-component reading of the same
    # texels (n_z = 0) renders differently
    sc.set_normal_encoding("xyz")
    out3, _ = P.render(sc, cam)
    torch.cuda.synchronize()
    assert np.abs(out3.cpu().numpy() - out.cpu().numpy()).max() > 1e-2
    saved.release()


def test_xy_hw_and_flat_samplers_on_constant_charts(P):
    scene = xy_scene(const=True, n=1000)
    env = sg.make_env(0)
    cam = sg.look_at_camera((3.2, 1.0, 0.8), 128, 128)
    sc = P.Scene.from_arrays(scene, env)
    sc.build_atlas2d("f32")
    imgs = {}
    for smp in ("software", "hw_atlas", "flat"):
        sc.set_sampler(smp)
        o, _ = P.render(sc, cam)
        torch.cuda.synchronize()
        imgs[smp] = o.cpu().numpy().astype(np.float64)
    assert np.abs(imgs["hw_atlas"] - imgs["software"]).max() <= 1e-5
    assert np.abs(imgs["flat"] - imgs["software"]).max() <= 1e-5
    rng = np.random.default_rng(1)
    px, py = rng.integers(0, 128, 300), rng.integers(0, 128, 300)
    ref = R.render_pixels(scene, cam, env, px, py)
    check_admissible(imgs["software"][py, px], ref, 1e-4, 1e-3, "two-component normals, sampled")


def test_mixed_encodings_in_one_batch_are_rejected(P):
    env = sg.make_env(0, cube_res=8, levels=1, irr_res=4, lut_res=16)
    a = P.Scene.from_arrays(sg.make_scene(0, n=64, T=4, seed=1), env)
    b = P.Scene.from_arrays(xy_scene(n=64), env)
    cam = sg.look_at_camera((4.0, 0.0, 0.0), 32, 32)
    with pytest.raises(P.TexSplatError, match="TS_ERR_ARG"):
        P.render_views([a, b], [cam, cam])


@pytest.mark.parametrize("with_sh", [False, True])
def test_xy_gradients_match_oracle(P, with_sh):
    scene = xy_scene(seed=5)
    if with_sh:
        rng = np.random.default_rng(6)
        scene["sh"] = (rng.normal(size=(600, 9, 3)) * 0.3).astype(np.float32)
    env = sg.make_env(5, cube_res=16, levels=2, irr_res=8, lut_res=32)
    cam = sg.look_at_camera((2.6, 1.2, 0.8), 96, 80)
    H, W = 80, 96
    vis = np.random.default_rng(7).uniform(0, 1, size=(H, W)).astype(np.float32) if with_sh else None
    kl = K.build_keys(scene, cam)
    ref_fwd = R.render(scene, cam, env, keylist=kl, vis=vis)
    gamb = ref_fwd["grad_ambiguous"].numpy()
    assert gamb.mean() < 0.03
    rng = np.random.default_rng(9)
    dL = rng.normal(size=(H, W, 4))
    dL[gamb] = 0.0
    ref = G.render_grads(scene, cam, env, dL, keylist=kl, vis=vis)
    sc = P.Scene.from_arrays(scene, env)
    cg = dict(cam, vis=torch.from_numpy(vis).cuda()) if with_sh else cam
    _, saved = P.render(sc, cg, save=True)
    grads = P.zero_grads(sc)
    P.render_backward(saved, torch.from_numpy(dL.astype(np.float32)).cuda(), grads)
    torch.cuda.synchronize()
    names = ("means", "quats", "scales", "opacity", "texels") + (("sh",) if with_sh else ())
    for name in names:
        r = ref[name]
        g = grads[name].cpu().numpy().astype(np.float64).reshape(r.shape)
        scale = np.abs(r).max()
        assert scale > 0, name
        err = np.abs(g - r)
        bad = err > 1e-3 * scale + 1e-6
        assert not bad.any(), (name, int(bad.sum()), float(err.max()), float(scale))
    gt = grads["texels"].cpu().numpy()
    assert np.abs(gt[..., 7]).max() == 0.0
    saved.release()


@pytest.mark.parametrize("store,tdt", [("bf16", torch.bfloat16), ("f16", torch.float16)])
def test_reduced_precision_atlas_with_both_features(P, store, tdt):
    """BF16 / F16 atlases with two-component normals and indirect light:
    image and gradients against the oracle fed the same rounded texels."""
    scene = xy_scene(seed=8)
    rounded = torch.from_numpy(scene["texels"]).to(tdt).to(torch.float32).numpy()
    rng = np.random.default_rng(12)
    scene["sh"] = (rng.normal(size=(600, 4, 3)) * 0.3).astype(np.float32)
    env = sg.make_env(6, cube_res=16, levels=2, irr_res=8, lut_res=32)
    cam = sg.look_at_camera((2.6, 1.2, 0.8), 96, 80)
    H, W = 80, 96
    vis = rng.uniform(0, 1, size=(H, W)).astype(np.float32)
    ref_scene = dict(scene, texels=rounded)
    kl = K.build_keys(ref_scene, cam)
    ref = R.render(ref_scene, cam, env, keylist=kl, vis=vis)
    sc = P.Scene.from_arrays(scene, env, store=store)
    cg = dict(cam, vis=torch.from_numpy(vis).cuda())
    out, saved = P.render(sc, cg, save=True)
    torch.cuda.synchronize()
    check_admissible(out.cpu().numpy(), ref, 1e-4, 1e-3, f"indirect + two-component normals, {store}")
    gamb = ref["grad_ambiguous"].numpy()
    dL = np.random.default_rng(13).normal(size=(H, W, 4))
    dL[gamb] = 0.0
    rg = G.render_grads(ref_scene, cam, env, dL, keylist=kl, vis=vis)
    grads = P.zero_grads(sc)
    P.render_backward(saved, torch.from_numpy(dL.astype(np.float32)).cuda(), grads)
    torch.cuda.synchronize()
    for name in ("means", "quats", "scales", "opacity", "texels", "sh"):
        r = rg[name]
        g = grads[name].cpu().numpy().astype(np.float64).reshape(r.shape)
        scale = np.abs(r).max()
        bad = np.abs(g - r) > 1e-3 * scale + 1e-6
        assert not bad.any(), (name, int(bad.sum()), float(np.abs(g - r).max()), float(scale))
    saved.release()


def test_features_on_edge_cases(P):
    """Both features on: an empty scene, a fully culled scene (zero image,
    zero gradients) and a single splat on a ragged 17 x 13 image (oracle)."""
    env = sg.make_env(0, cube_res=8, irr_res=4, lut_res=16)
    cam = sg.look_at_camera((4.0, 0.0, 0.0), 40, 24)
    empty = dict(means=np.zeros((0, 3), np.float32), quats=np.zeros((0, 4), np.float32),
                 scales=np.zeros((0, 2), np.float32), opacity=np.zeros(0, np.float32),
                 texels=np.zeros((0, 4, 4, 8), np.float32), T=4, sh=np.zeros((0, 9, 3), np.float32),
                 normal_encoding="xy")
    vis = torch.full((24, 40), 0.5, device="cuda")
    sc = P.Scene.from_arrays(empty, env)
    out, saved = P.render(sc, dict(cam, vis=vis), save=True)
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0
    saved.release()
    # every splat behind the camera
    culled = xy_scene(n=50)
    culled["means"][:, 0] += 10.0
    culled["sh"] = np.ones((50, 4, 3), np.float32)
    sc = P.Scene.from_arrays(culled, env)
    out, saved = P.render(sc, dict(cam, vis=vis), save=True)
    grads = P.zero_grads(sc)
    P.render_backward(saved, torch.ones(24, 40, 4, device="cuda"), grads)
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0
    for k in ("means", "texels", "sh"):
        assert torch.count_nonzero(grads[k]).item() == 0
    saved.release()
    # one splat, ragged image
    one = xy_scene(n=1, seed=9)
    one["means"][:] = 0.0
    one["scales"][:] = 0.4
    one["opacity"][:] = 0.9
    one["sh"] = (np.random.default_rng(4).normal(size=(1, 9, 3)) * 0.3).astype(np.float32)
    cam1 = sg.look_at_camera((3.0, 0.4, 0.2), 17, 13)
    v1 = np.random.default_rng(5).uniform(0, 1, size=(13, 17)).astype(np.float32)
    ref = R.render(one, cam1, env, vis=v1)
    sc = P.Scene.from_arrays(one, env)
    out, _ = P.render(sc, dict(cam1, vis=torch.from_numpy(v1).cuda()))
    torch.cuda.synchronize()
    assert (ref["A"].numpy() > 0).sum() > 20
    check_admissible(out.cpu().numpy(), ref, 1e-4, 1e-3, "one splat, ragged")
