"""Pins of the FP32 binning/sort specification (oracle/keys.py)."""
import numpy as np
from scipy.spatial.transform import Rotation

import scenegen as sg
from oracle import keys as K
from oracle import render as R
from tests.helpers import cam_identity, fronto_scene


def fp64_corners_px(scene, cam):
    """Projected 3-sigma corners in float64 with a library rotation (scipy)."""
    q = scene["quats"].astype(np.float64)
    rot = Rotation.from_quat(np.concatenate([q[:, 1:], q[:, :1]], 1)).as_matrix()
    tu, tv = rot[:, :, 0], rot[:, :, 1]
    p = scene["means"].astype(np.float64)
    s = scene["scales"].astype(np.float64)
    out = []
    for a, b in [(-1, -1), (1, -1), (-1, 1), (1, 1)]:
        c = p + a * 3 * s[:, :1] * tu + b * 3 * s[:, 1:] * tv
        Xc = c @ cam["R"].astype(np.float64).T + cam["t"].astype(np.float64)
        out.append(np.stack([cam["fx"] * Xc[:, 0] / Xc[:, 2] + cam["cx"],
                             cam["fy"] * Xc[:, 1] / Xc[:, 2] + cam["cy"], Xc[:, 2]], -1))
    return np.stack(out, 1)


def test_rotation_columns_match_library_rotation():
    scene = sg.make_scene(1, n=2000, T=1, seed=3)
    tu, tv, n = K.rotation_columns_f32(scene["quats"] * np.float32(1.7))  # unnormalised input
    q = scene["quats"].astype(np.float64)
    rot = Rotation.from_quat(np.concatenate([q[:, 1:], q[:, :1]], 1)).as_matrix()
    np.testing.assert_allclose(tu, rot[:, :, 0], atol=1e-6)
    np.testing.assert_allclose(tv, rot[:, :, 1], atol=1e-6)
    np.testing.assert_allclose(n, rot[:, :, 2], atol=1e-6)
    np.testing.assert_allclose(np.cross(tu, tv), n, atol=1e-6)


def test_fp32_corners_match_fp64_projection():
    scene = sg.make_scene(1, n=5000, T=1, seed=4)
    cam = sg.fibonacci_cameras(7, 4.0, 800, 800)[3]
    sv = K.splat_view_f32(scene, cam)
    ref = fp64_corners_px(scene, cam)
    vis = sv["visible"]
    assert vis.sum() > 4000
    err = np.abs(sv["corners_px"][vis] - ref[vis][..., :2]).max()
    assert err < 5e-3, err


def test_rect_covers_every_contributing_pixel():
    # a pixel is covered only inside the projected support square; every such
    # pixel centre found by the FP64 renderer must lie in the splat's tile rect
    scene = sg.make_scene(0, n=96, T=4, seed=21)
    cam = sg.look_at_camera((2.2, 1.4, 0.3), 96, 80)
    env = sg.make_env(0, cube_res=8, irr_res=4, lut_res=16)
    kl = K.build_keys(scene, cam)
    out = R.render(scene, cam, env, brute=True)
    # recover the blended (pixel, splat) pairs from the brute-force lists
    import torch
    params = R.to_params(scene)
    cand = R.brute_candidates(kl["view"])
    H, W = 80, 96
    gy, gx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    fr = R.fragments(params, cam, gx.ravel(), gy.ravel(),
                     torch.from_numpy(np.broadcast_to(cand, (H * W, cand.size)).copy()))
    pix, which = np.nonzero(fr["blended"].numpy())
    k = cand[which]
    tx, ty = gx.ravel()[pix] // 16, gy.ravel()[pix] // 16
    rect = kl["view"]["rect"][k]
    assert ((rect[:, 0] <= tx) & (tx <= rect[:, 1]) & (rect[:, 2] <= ty) & (ty <= rect[:, 3])).all()
    assert pix.size > 1000
    assert out["A"].numpy().max() > 0


def test_key_order_and_tie_break():
    scene = sg.make_scene(0, seed=0)
    cam = sg.look_at_camera((4.0, 0.0, 0.0), 128, 128)
    kl = K.build_keys(scene, cam)
    keys, ids = kl["keys"], kl["ids"]
    assert np.all(keys[1:] >= keys[:-1])
    same = keys[1:] == keys[:-1]
    assert np.all(ids[1:][same] > ids[:-1][same])
    # identical depths: two splats at the same centre keep id order
    tex = np.zeros((3, 2, 2, 8), np.float32)
    sc = fronto_scene([[0, 0, 1.0], [0.1, 0, 1.0], [0, 0, 1.0]], [[0.1, 0.1]] * 3, [0.5] * 3, tex)
    kl2 = K.build_keys(sc, cam_identity())
    t = kl2["tile_ranges"][(64 // 16) * 8 + 64 // 16]
    lst = kl2["ids"][t[0]:t[1]].tolist()
    assert lst.index(0) < lst.index(2)


def test_culling_rules():
    tex = np.zeros((4, 2, 2, 8), np.float32)
    sc = fronto_scene([[0, 0, 1.0],      # visible
                       [0, 0, 0.21],     # corners at z = 0.21 > 0.2 but huge on screen -> visible
                       [0, 0, 1.0],      # opacity below 1/255 -> culled
                       [0.5, 0.0, 0.3]], # tilted below: give it a rotation so a corner is behind the near plane
                      [[0.1, 0.1], [0.01, 0.01], [0.1, 0.1], [0.1, 0.1]],
                      [0.5, 0.5, 0.0039, 0.5], tex)
    # rotate splat 3 by 90 deg about x so its v axis points along z: corners at
    # z = 0.3 +- 0.3 -> one side at z = 0 <= 0.2 -> culled
    c, s = np.cos(np.pi / 4), np.sin(np.pi / 4)
    sc["quats"][3] = [c, s, 0, 0]
    sv = K.splat_view_f32(sc, cam_identity())
    assert sv["visible"].tolist() == [True, True, False, False]
    # out-of-image splat: empty tile rect -> culled
    sc2 = fronto_scene([[50.0, 0, 1.0]], [[0.1, 0.1]], [0.5], tex[:1])
    assert not K.splat_view_f32(sc2, cam_identity())["visible"][0]


def test_tile_rect_formula_closed_form():
    # fronto splat at depth 1: corners at x = 64 (X0 +- 3 s_u) + 64
    tex = np.zeros((1, 2, 2, 8), np.float32)
    sc = fronto_scene([[0.25, -0.125, 1.0]], [[0.0625, 0.125]], [0.5], tex)
    sv = K.splat_view_f32(sc, cam_identity())
    xmin, xmax = 64 * (0.25 - 0.1875) + 64, 64 * (0.25 + 0.1875) + 64
    ymin, ymax = 64 * (-0.125 - 0.375) + 64, 64 * (-0.125 + 0.375) + 64
    assert sv["rect"][0].tolist() == [int(xmin // 16), int(xmax // 16), int(ymin // 16), int(ymax // 16)]
    kl = K.build_keys(sc, cam_identity())
    nt = (int(xmax // 16) - int(xmin // 16) + 1) * (int(ymax // 16) - int(ymin // 16) + 1)
    assert kl["keys"].size == nt
    assert np.all((kl["keys"] & np.uint64(0xFFFFFFFF)) == np.float32(1.0).view(np.uint32))
