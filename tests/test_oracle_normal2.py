"""Pins of the oracle's two-component tangent-normal encoding (Sec. 3.5.1:
n_z = sqrt(max(0, 1 - n_x^2 - n_y^2)) rebuilt at render time): a closed form
for a fronto-parallel splat with a linear (n_x, n_y) texture, the clamp
outside the unit disc, the equivalence with three stored components for
per-splat constant normals, and central differences of the gradient."""
import math

import numpy as np

import scenegen as sg
from oracle import grad as G
from oracle import keys as K
from oracle import render as R
from tests.helpers import cam_identity, fronto_scene


def linear_normal_splat(nx0=0.1, bx=0.05, ny0=-0.2, by=0.1, T=4):
    """One fronto-parallel splat at depth 2 whose texel (i, j) stores
    n_x = nx0 + bx i, n_y = ny0 + by j (channel 7 left at zero)."""
    tex = np.zeros((1, T, T, 8), dtype=np.float32)
    tex[..., 0:3] = 0.5
    tex[..., 3] = 0.1
    tex[..., 4] = 0.6
    for j in range(T):
        for i in range(T):
            tex[0, j, i, 5] = nx0 + bx * i
            tex[0, j, i, 6] = ny0 + by * j
    sc = fronto_scene([[0.0, 0.0, 2.0]], [[0.5, 0.5]], [0.9], tex)
    return sc


def test_rebuilt_normal_of_a_linear_texture_in_closed_form():
    sc = linear_normal_splat()
    sc["normal_encoding"] = "xy"
    cam = cam_identity(W=48, H=48, f=30.0, cx=24.0, cy=24.0)
    out = R.render(sc, cam, sg.constant_env((0.5, 0.5, 0.5)))
    X, A = out["X"].numpy(), out["A"].numpy()
    T = 4
    checked = 0
    for y in range(48):
        for x in range(48):
            if A[y, x] <= 0:
                continue
            # ray (x', y', 1)/f hits z = 2: u = 2 x' / (f s), identity frame
            dx = (x + 0.5 - 24.0) / 30.0
            dy = (y + 0.5 - 24.0) / 30.0
            u, v = 2.0 * dx / float(np.float32(0.5)), 2.0 * dy / float(np.float32(0.5))
            cs, ct = (u + 3.0) / 6.0 * T - 0.5, (v + 3.0) / 6.0 * T - 0.5
            if not (0.0 <= cs <= T - 1 and 0.0 <= ct <= T - 1):
                continue  # clamp-to-edge region: not linear
            # bilinear interpolation of a linear function is that function
            nx = float(np.float32(0.1)) + float(np.float32(0.05)) * cs
            ny = float(np.float32(-0.2)) + float(np.float32(0.1)) * ct
            nz = math.sqrt(max(0.0, 1.0 - nx * nx - ny * ny))
            # t_u = x, t_v = y, the splat normal +z turned to face the camera
            expect = np.array([nx, ny, -nz])
            np.testing.assert_allclose(X[y, x, 5:8] / A[y, x], expect, atol=2e-8)
            checked += 1
    assert checked > 300
    # three stored components with the per-texel n_z interpolate n_z itself,
    # which differs (the rebuild is not linear): the test sees the encoding
    sc3 = linear_normal_splat()
    t = sc3["texels"]
    t[..., 7] = np.sqrt(np.maximum(0.0, 1.0 - t[..., 5] ** 2 - t[..., 6] ** 2))
    out3 = R.render(sc3, cam, sg.constant_env((0.5, 0.5, 0.5)))
    assert np.abs(out3["X"].numpy()[..., 7] - X[..., 7]).max() > 1e-6


def test_rebuilt_normal_is_clamped_outside_the_unit_disc():
    sc = linear_normal_splat(nx0=0.9, bx=0.0, ny0=0.9, by=0.0)
    sc["normal_encoding"] = "xy"
    cam = cam_identity(W=32, H=32, f=20.0, cx=16.0, cy=16.0)
    out = R.render(sc, cam, sg.constant_env((0.5, 0.5, 0.5)))
    X, A = out["X"].numpy(), out["A"].numpy()
    m = A > 0
    assert m.sum() > 100
    n = X[m][:, 5:8] / A[m][:, None]
    f = float(np.float32(0.9))
    np.testing.assert_allclose(n, np.broadcast_to([f, f, 0.0], n.shape), atol=1e-12)


def constant_normal_scene(seed=2):
    scene = sg.make_scene(0, n=300, T=4, seed=seed)
    rng = np.random.default_rng(seed)
    n = rng.normal(size=(300, 3)) * np.array([0.3, 0.3, 0.0]) + np.array([0.0, 0.0, 1.0])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    tex = scene["texels"]
    tex[..., 5:8] = n[:, None, None, :].astype(np.float32)
    # the two-component scene stores n_x, n_y only; its n_z is rebuilt, so
    # the three-component scene gets the rebuilt value of the stored pair
    nx, ny = tex[..., 5].astype(np.float64), tex[..., 6].astype(np.float64)
    s3 = dict(scene, texels=tex.copy())
    s3["texels"][..., 7] = np.sqrt(1.0 - nx * nx - ny * ny).astype(np.float32)
    s2 = dict(scene, texels=tex.copy(), normal_encoding="xy")
    s2["texels"][..., 7] = 0.0
    return s2, s3


def test_constant_normals_render_as_three_components():
    s2, s3 = constant_normal_scene()
    cam = sg.look_at_camera((4.0, 0.5, 0.3), 64, 64)
    env = sg.make_env(1, cube_res=8, levels=2, irr_res=4, lut_res=16)
    kl = K.build_keys(s3, cam)
    o2 = R.render(s2, cam, env, keylist=kl)
    o3 = R.render(s3, cam, env, keylist=kl)
    assert (o3["A"].numpy() > 0.1).sum() > 500
    # n_z of s3 is float32-rounded, s2 rebuilds it in float64: ~6e-8 apart
    assert np.abs(o2["X"].numpy() - o3["X"].numpy()).max() <= 1e-6
    assert np.abs(o2["rgba"].numpy() - o3["rgba"].numpy()).max() <= 1e-5


def test_two_component_gradient_matches_central_differences():
    scene = sg.make_scene(0, n=48, T=4, seed=13)
    scene["texels"][..., 7] = 0.0
    scene["normal_encoding"] = "xy"
    cam = sg.look_at_camera((3.0, 0.8, 0.4), 48, 48)
    env = sg.make_env(4, cube_res=8, levels=2, irr_res=4, lut_res=16)
    rng = np.random.default_rng(5)
    dL = rng.normal(size=(48, 48, 4))
    kl = K.build_keys(scene, cam)
    gr = G.render_grads(scene, cam, env, dL, keylist=kl)
    gt = gr["texels"]
    # channel 7 is not read
    assert np.abs(gt[..., 7]).max() == 0.0
    scale = np.abs(gt[..., 5:7]).max()
    assert scale > 0
    for c in (5, 6):
        flat = np.argsort(-np.abs(gt[..., c]).ravel())[:4]
        for fi in flat:
            idx = np.unravel_index(fi, gt[..., c].shape) + (c,)
            fd = G.central_difference(scene, cam, env, dL, "texels", idx, 1e-7, keylist=kl)
            assert abs(fd - gt[idx]) <= 1e-5 * scale + 1e-6 * abs(fd), (idx, fd, gt[idx])
    for name in ("means", "quats"):
        g = gr[name]
        idx = np.unravel_index(int(np.argmax(np.abs(g))), g.shape)
        fd = G.central_difference(scene, cam, env, dL, name, idx, 1e-7, keylist=kl)
        assert abs(fd - g[idx]) <= 1e-5 * np.abs(g).max() + 1e-6 * abs(fd), (name, idx, fd, g[idx])
