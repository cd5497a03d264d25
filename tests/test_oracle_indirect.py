"""Pins of the oracle's indirect light (per-splat SH evaluated in each
fragment's reflection direction, blended, mixed into the specular term by a
visibility V: Eq. 9 and Eq. 12 with L_ind)."""
import math

import numpy as np
import torch

import scenegen as sg
from oracle import grad as G
from oracle import keys as K
from oracle import render as R
from oracle import shading as S
from tests.helpers import cam_identity, fronto_scene

ENV_C = np.array([0.7, 0.5, 0.3], dtype=np.float32)
LUT_AB = (0.625, 0.125)


def test_sh_basis_is_orthonormal():
    # product quadrature exact for polynomials of degree <= 4 on the sphere
    xg, wg = np.polynomial.legendre.leggauss(16)
    phi = (np.arange(32) + 0.5) * 2 * math.pi / 32
    ct, ph = np.meshgrid(xg, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    w = torch.tensor(np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1))
    Y = S.sh_basis(w, 9).numpy()  # [16, 32, 9]
    wts = (wg[:, None] * np.full(32, 2 * math.pi / 32)[None, :])
    gram = np.einsum("ijk,ijl,ij->kl", Y, Y, wts)
    np.testing.assert_allclose(gram, np.eye(9), atol=1e-12)


def one_splat(sh):
    attr = np.array([0.2, 0.6, 0.9, 0.3, 0.4, 0.0, 0.0, 1.0], dtype=np.float32)
    tex = np.broadcast_to(attr, (1, 4, 4, 8)).copy()
    sc = fronto_scene([[0.05, -0.03, 1.0]], [[0.15, 0.2]], [0.9], tex)
    sc["sh"] = np.asarray(sh, dtype=np.float32)[None]
    return sc, attr


def closed_form(attr, A, lind, vis, env):
    alb, met = attr[:3].astype(np.float64), float(attr[3])
    f0 = 0.04 * (1.0 - met) + alb * met
    c = env["spec"][0][0, 0, 0].astype(np.float64)            # radiance
    e = env["irr"][0, 0, 0].astype(np.float64) / math.pi      # irradiance / pi as stored
    spec = vis[..., None] * c + (1.0 - vis[..., None]) * lind
    return A[..., None] * (alb * (1.0 - met) * e + (f0 * LUT_AB[0] + LUT_AB[1]) * spec)


def test_visibility_one_leaves_the_image_unchanged():
    rng = np.random.default_rng(0)
    sc, _ = one_splat(rng.normal(size=(9, 3)))
    cam = cam_identity()
    env = sg.constant_env(ENV_C, lut=LUT_AB)
    base = R.render({k: v for k, v in sc.items() if k != "sh"}, cam, env)
    withsh = R.render(sc, cam, env, vis=np.ones((128, 128)))
    np.testing.assert_allclose(withsh["rgba"].numpy(), base["rgba"].numpy(), atol=1e-15)


def test_indirect_light_closed_form_single_splat():
    """V < 1 with a flat normal map: every fragment's normal is the splat
    normal turned to the camera, n = (0, 0, -1); the reflection of
    w_o = -d/|d| is w_r = 2 (n . w_o) n - w_o and the indirect light is
    c . Y(w_r) per channel."""
    rng = np.random.default_rng(1)
    sh = rng.normal(size=(9, 3))
    sc, attr = one_splat(sh)
    cam = cam_identity()
    env = sg.constant_env(ENV_C, lut=LUT_AB)
    vis = rng.uniform(size=(128, 128))
    out = R.render(sc, cam, env, vis=vis)
    A = out["A"].numpy()
    xs = (np.arange(128) + 0.5 - 64.0) / 64.0
    d = np.stack(np.broadcast_arrays(xs[None, :], xs[:, None], np.ones((128, 128))), -1)
    wo = -d / np.linalg.norm(d, axis=-1, keepdims=True)
    n = np.array([0.0, 0.0, -1.0])
    wr = 2 * (wo @ n)[..., None] * n - wo
    Y = S.sh_basis(torch.tensor(wr), 9).numpy()
    lind = Y @ sh.astype(np.float32).astype(np.float64)
    m = A > 0
    assert m.sum() > 300
    np.testing.assert_allclose(out["Xind"].numpy()[m], A[m][:, None] * lind[m], atol=1e-13)
    col = closed_form(attr, A, lind, vis, env)
    np.testing.assert_allclose(out["rgba"].numpy()[..., :3][m], col[m], atol=1e-12)


def test_indirect_gradients_match_central_differences():
    sc = sg.make_scene(0, n=40, T=4, seed=5)
    rng = np.random.default_rng(2)
    sc["sh"] = (rng.normal(size=(40, 9, 3)) * 0.3).astype(np.float32)
    cam = sg.look_at_camera((3.2, 0.4, 0.3), 40, 40)
    env = sg.make_env(0, cube_res=8, irr_res=4, lut_res=16)
    vis = rng.uniform(0.0, 0.6, size=(40, 40))
    kl = K.build_keys(sc, cam)
    dL = rng.normal(size=(40, 40, 4))
    g = G.render_grads(sc, cam, env, dL, keylist=kl, vis=vis)
    assert np.abs(g["sh"]).max() > 0
    nz = np.argwhere(np.abs(g["sh"]) > 1e-3 * np.abs(g["sh"]).max())
    for idx in [tuple(nz[i]) for i in (0, len(nz) // 2, len(nz) - 1)]:
        fd = G.central_difference(sc, cam, env, dL, "sh", idx, 1e-6, keylist=kl, vis=vis)
        np.testing.assert_allclose(g["sh"][idx], fd, rtol=1e-6, atol=1e-9)
    # a tangent-normal texel: the reflection direction depends on it
    idx = tuple(np.argwhere(np.abs(g["texels"][..., 5]) > 0)[0]) + ()
    idx = (idx[0], idx[1], idx[2], 5)
    fd = G.central_difference(sc, cam, env, dL, "texels", idx, 1e-6, keylist=kl, vis=vis)
    np.testing.assert_allclose(g["texels"][idx], fd, rtol=1e-5, atol=1e-9)
