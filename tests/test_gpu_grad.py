"""Gradients of the CUDA backward (through the C ABI) against the FP64
oracle's autograd gradients of the same forward.

Bar per element: |g_gpu - g_ref| <= 1e-3 * max|g_ref| + 1e-6 within each
parameter group.  The upstream gradient is zeroed on pixels the oracle flags
as gradient-ambiguous: a threshold decision there may differ between FP32
and FP64, or the pixel sits within FP32 error of a derivative kink (a
bilinear cell boundary of a texture, the BRDF table or a cube map, the
opacity clamp), where the value is continuous but the slope is not.
"""
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
    return P


def run_case(P, scene, env, cam, seed=0, store="f32"):
    kl = K.build_keys(scene, cam)
    ref_fwd = R.render(scene, cam, env, keylist=kl)
    amb = ref_fwd["grad_ambiguous"].numpy()
    assert amb.mean() < 0.02, amb.mean()
    rng = np.random.default_rng(seed)
    H, W = int(cam["H"]), int(cam["W"])
    dL = rng.normal(size=(H, W, 4))
    dL[amb] = 0.0
    ref = G.render_grads(scene, cam, env, dL, keylist=kl)
    sc = P.Scene.from_arrays(scene, env, store=store)
    out, saved = P.render(sc, cam, save=True)
    grads = P.zero_grads(sc)
    P.render_backward(saved, torch.from_numpy(dL.astype(np.float32)).cuda(), grads)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}
    spec_ref = np.concatenate([s.ravel() for s in ref["spec"]])
    pairs = [("means", got["means"], ref["means"]), ("quats", got["quats"], ref["quats"]),
             ("scales", got["scales"], ref["scales"]), ("opacity", got["opacity"], ref["opacity"]),
             ("texels", got["texels"], ref["texels"]), ("spec", got["spec"], spec_ref),
             ("irr", got["irr"], ref["irr"].ravel())]
    report = {}
    for name, g, r in pairs:
        g = g.reshape(r.shape)
        scale = np.abs(r).max()
        err = np.abs(g - r)
        tol = 1e-3 * scale + 1e-6
        report[name] = (float(err.max()), float(scale))
        bad = err > tol
        assert not bad.any(), (name, int(bad.sum()), float(err.max()), float(scale), np.argwhere(bad)[:5])
    return report


def test_grad_parity_cfg0(P):
    scene = sg.make_scene(0)
    env = sg.make_env(0, cube_res=16, levels=2, irr_res=8, lut_res=32)
    cam = sg.look_at_camera((4.0, 0.0, 0.0), 128, 128)
    run_case(P, scene, env, cam, seed=1)


def test_grad_parity_ragged_view(P):
    scene = sg.make_scene(1, n=500, T=4, seed=6)
    env = sg.make_env(6, cube_res=8, levels=3, irr_res=4, lut_res=16)
    cam = sg.look_at_camera((2.0, 2.2, 0.7), 90, 70)
    run_case(P, scene, env, cam, seed=2)


def test_grad_parity_bf16_atlas(P):
    scene = sg.make_scene(0, n=200, T=8, seed=7)
    scene["texels"] = torch.from_numpy(scene["texels"]).to(torch.bfloat16).float().numpy()
    env = sg.make_env(7, cube_res=8, irr_res=4, lut_res=16)
    cam = sg.look_at_camera((3.0, -1.0, 0.5), 80, 80)
    run_case(P, scene, env, cam, seed=3, store="bf16")


@pytest.mark.parametrize("T", [1, 32])
def test_grad_parity_texture_resolution_limits(P, T):
    """The smallest (one texel: per-splat attributes) and the largest
    texture resolution the ABI accepts."""
    scene = sg.make_scene(1, n=300, T=T, seed=10 + T)
    env = sg.make_env(8, cube_res=8, levels=2, irr_res=4, lut_res=16)
    cam = sg.look_at_camera((2.4, -1.2, 0.9), 72, 60)
    kl = K.build_keys(scene, cam)
    sc = P.Scene.from_arrays(scene, env)
    out, _ = P.render(sc, cam)
    torch.cuda.synchronize()
    ref = R.render(scene, cam, env, keylist=kl)
    check_admissible(out.cpu().numpy(), ref, 1e-4, 1e-3, f"T={T}")
    run_case(P, scene, env, cam, seed=4)


def test_batch_of_the_maximum_view_count_equals_alone_renders(P):
    scene = sg.make_scene(1, n=2000, T=4, seed=12)
    env = sg.make_env(9, cube_res=8, irr_res=4, lut_res=16)
    cams = [sg.look_at_camera(tuple(np.asarray(c["R"]).T @ -np.asarray(c["t"])), 24 + (i % 5) * 7, 20 + (i % 3) * 9)
            for i, c in enumerate(sg.fibonacci_cameras(32, 3.5, 8, 8))]
    sc = P.Scene.from_arrays(scene, env)
    outs, _ = P.render_views([sc] * 32, cams)
    for c, o in zip(cams, outs):
        a, _ = P.render(sc, c)
        torch.cuda.synchronize()
        assert torch.equal(a, o)
    with pytest.raises(P.TexSplatError, match="TS_ERR_ARG"):
        P.render_views([sc] * 33, cams + cams[:1])


def test_batched_backward_equals_the_sum_of_view_backwards(P):
    """One launch sequence over four views (the training bench's step):
    images bit-identical to the views rendered alone, and the accumulated
    gradients equal the sum of the four single-view backwards up to the
    order of the atomic additions (1e-4 of each group's maximum)."""
    scene = sg.make_scene(1, n=20000, T=8, seed=21)
    env = sg.make_env(1, cube_res=16, levels=1, irr_res=8, lut_res=32)
    cams = sg.fibonacci_cameras(4, 4.0, 192, 160)
    sc = P.Scene.from_arrays(scene, env)
    rng = np.random.default_rng(3)
    dls = [torch.from_numpy(rng.normal(size=(160, 192, 4)).astype(np.float32)).cuda() for _ in cams]
    outs, saved = P.render_views([sc] * 4, cams, save=True)
    g_batch = P.zero_grads(sc)
    P.render_backward(saved, dls, g_batch)
    saved.release()
    g_sum = P.zero_grads(sc)
    for c, d, o in zip(cams, dls, outs):
        a, sv = P.render(sc, c, save=True)
        P.render_backward(sv, d, g_sum)
        sv.release()
        torch.cuda.synchronize()
        assert torch.equal(a, o)
    torch.cuda.synchronize()
    for k in g_batch:
        a, b = g_batch[k].double(), g_sum[k].double()
        scale = float(b.abs().max())
        assert scale > 0.0, k
        err = float((a - b).abs().max())
        print(f"[batch] {k}: max |batched - summed| {err:.3g} of max {scale:.3g}")
        assert err <= 1e-4 * scale + 1e-9, (k, err, scale)
