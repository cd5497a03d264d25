"""Hardware-texture atlas sampler (supplementary Sec. 1) and the flat
(untextured) sampler against the software bilinear path.

The texture unit computes bilinear weights in fixed point with 8 fractional
bits, so the hardware path is a reported-error path: it must agree with the
software path exactly where the filter cannot matter (constant charts, the
alpha channel) and within the weight quantisation where it does.
"""
import numpy as np
import pytest
import torch

import scenegen as sg
from oracle import render as R
from tests.helpers import check_admissible

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2506_13348_b300 as P
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return P


def scene_1k(T=8, const=False, metal_zero=False, n=1000):
    scene = sg.make_scene(1, n=n, T=T, seed=7)
    tex = scene["texels"]
    if const:
        tex[:] = tex[:, :1, :1, :]
    if metal_zero:
        tex[..., 3] = 0.0
    scene["texels"] = np.ascontiguousarray(tex)
    return scene


CAM = sg.look_at_camera((3.2, 1.0, 0.8), 256, 256)


def render(P, sc, sampler):
    sc.set_sampler(sampler)
    out, _ = P.render(sc, CAM)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def test_constant_charts_hw_and_flat_equal_software(P):
    scene = scene_1k(const=True)
    env = sg.make_env(0)
    sc = P.Scene.from_arrays(scene, env)
    sc.build_atlas2d("f32")
    sw = render(P, sc, "software")
    hw = render(P, sc, "hw_atlas")
    flat = render(P, sc, "flat")
    assert np.abs(sw).max() > 0.05
    assert np.abs(hw - sw).max() <= 1e-5, np.abs(hw - sw).max()
    assert np.abs(flat - sw).max() <= 1e-5, np.abs(flat - sw).max()
    # and the flat renderer is the oracle's per-splat-attribute image
    rng = np.random.default_rng(3)
    px, py = rng.integers(0, 256, 300), rng.integers(0, 256, 300)
    ref = R.render_pixels(scene, CAM, env, px, py)
    check_admissible(flat[py, px], ref, 1e-4, 1e-3, "flat sampler vs oracle")


def test_hw_sampler_within_weight_quantisation(P):
    """Metallic 0 and a constant environment make the colour affine in the
    blended albedo: colour = c (X_albedo + 0.04 A) with LUT (1, 0).  The
    albedo error of one hardware sample is at most 2 axes x 2^-8 x the texel
    range (1), so |colour_hw - colour_sw| <= c 2^-7."""
    c = 0.8
    scene = scene_1k(metal_zero=True)
    env = sg.constant_env((c, c, c))
    sc = P.Scene.from_arrays(scene, env)
    sc.build_atlas2d("f32")
    sw = render(P, sc, "software")
    hw = render(P, sc, "hw_atlas")
    # alpha (coverage) does not depend on the textures: identical
    np.testing.assert_array_equal(hw[..., 3], sw[..., 3])
    d = np.abs(hw[..., :3] - sw[..., :3])
    assert d.max() <= c * 2.0 ** -7, d.max()
    assert d.max() > 0.0  # the hardware path really filtered in fixed point
    assert d.mean() <= c * 2.0 ** -10, d.mean()


def test_hw_sampler_textured_scene_and_f16_atlas(P):
    scene = scene_1k()
    env = sg.make_env(0)
    for store in ("f32", "f16"):
        sc = P.Scene.from_arrays(scene, env, store=store)
        sc.build_atlas2d(store)
        sw = render(P, sc, "software")
        hw = render(P, sc, "hw_atlas")
        np.testing.assert_array_equal(hw[..., 3], sw[..., 3])
        d = np.abs(hw - sw)
        assert d.max() <= 0.05, (store, d.max())
        assert d.mean() <= 2e-3, (store, d.mean())


def test_ragged_chart_rows_and_texture_sizes(P):
    """n not a multiple of the charts per atlas row; T = 2 and 16."""
    env = sg.make_env(0)
    for T, n in ((2, 777), (16, 301)):
        scene = scene_1k(T=T, const=True, n=n)
        sc = P.Scene.from_arrays(scene, env)
        sc.build_atlas2d("f32")
        sw = render(P, sc, "software")
        hw = render(P, sc, "hw_atlas")
        assert np.abs(hw - sw).max() <= 1e-5, (T, np.abs(hw - sw).max())


def test_sampler_state_errors(P):
    from paper_2506_13348_b300._lib import TexSplatError
    scene = scene_1k(n=200)
    env = sg.make_env(0)
    sc = P.Scene.from_arrays(scene, env)
    sc.set_sampler("hw_atlas")
    with pytest.raises(TexSplatError, match="TS_ERR_STATE"):
        P.render(sc, CAM)  # no 2-D atlas yet
    sc.build_atlas2d("f32")
    P.render(sc, CAM)
    with pytest.raises(TexSplatError, match="TS_ERR_STATE"):
        P.render(sc, CAM, save=True)  # inference-only sampler
    sc.upload_atlas(scene["texels"], "f32")
    with pytest.raises(TexSplatError, match="TS_ERR_STATE"):
        P.render(sc, CAM)  # stale after a texel upload
    sc.build_atlas2d("f32")
    P.render(sc, CAM)
    sc.set_sampler("flat")
    with pytest.raises(TexSplatError, match="TS_ERR_STATE"):
        P.render(sc, CAM, save=True)
    sc.set_sampler("software")
    _, saved = P.render(sc, CAM, save=True)
    saved.release()
    torch.cuda.synchronize()


def test_morton_packing_samples_the_same_texels(P):
    """Charts placed in the Morton order of the splat centres: the same texels
    are sampled (constant charts equal the software path; the albedo-linear
    scene stays within the fixed-point bound of the software path)."""
    env = sg.make_env(0)
    scene = scene_1k(const=True, n=1500)
    sc = P.Scene.from_arrays(scene, env)
    sc.build_atlas2d("f32", packing="morton")
    sw = render(P, sc, "software")
    hw = render(P, sc, "hw_atlas")
    assert np.abs(hw - sw).max() <= 1e-5
    c = 0.8
    scene = scene_1k(metal_zero=True, n=1500)
    sc = P.Scene.from_arrays(scene, sg.constant_env((c, c, c)))
    sw = render(P, sc, "software")
    sc.build_atlas2d("f32", packing="morton")
    hw_m = render(P, sc, "hw_atlas")
    sc.build_atlas2d("f32", packing="splat_id")
    hw_i = render(P, sc, "hw_atlas")
    for hw in (hw_m, hw_i):
        np.testing.assert_array_equal(hw[..., 3], sw[..., 3])
        assert np.abs(hw[..., :3] - sw[..., :3]).max() <= c * 2.0 ** -7
