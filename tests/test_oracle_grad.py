"""Pins of the oracle gradient (autograd of the FP64 forward) against central
finite differences of that forward, for every parameter group."""
import zlib

import numpy as np
import pytest

import scenegen as sg
from oracle import grad as G
from oracle import keys as K


@pytest.fixture(scope="module")
def setup():
    scene = sg.make_scene(0, n=48, T=4, seed=13)
    cam = sg.look_at_camera((3.0, 0.8, 0.4), 48, 48)
    env = sg.make_env(4, cube_res=8, levels=3, irr_res=4, lut_res=16)
    rng = np.random.default_rng(8)
    dL = rng.normal(size=(48, 48, 4))
    kl = K.build_keys(scene, cam)
    gr = G.render_grads(scene, cam, env, dL, keylist=kl)
    return scene, cam, env, dL, kl, gr


def _pick(gr, name, rng, k=3):
    g = gr[name] if not isinstance(name, tuple) else gr[name[0]][name[1]]
    flat = np.argsort(-np.abs(g).ravel())[: 4 * k]
    sel = rng.choice(flat, size=k, replace=False)
    return [np.unravel_index(i, g.shape) for i in sel], g


@pytest.mark.parametrize("name", ["means", "quats", "scales", "opacity", "texels", ("spec", 0),
                                  ("spec", 1), "irr"])
def test_autograd_matches_central_differences(setup, name):
    scene, cam, env, dL, kl, gr = setup
    rng = np.random.default_rng(zlib.crc32(str(name).encode()))
    idxs, g = _pick(gr, name, rng)
    scale = np.abs(g).max()
    assert scale > 0
    for idx in idxs:
        fd = G.central_difference(scene, cam, env, dL, name, idx, 1e-7, keylist=kl)
        assert abs(fd - g[idx]) <= 1e-5 * scale + 1e-6 * abs(fd), (name, idx, fd, g[idx])


def test_texel_gradients_of_a_constant_texture_sum_to_the_attribute_gradient():
    """With a constant texture the texel gradients of a splat, summed over
    its texels, are the gradient w.r.t. its per-splat attribute -- taken here
    by central differences of the separately written per-attribute 2DGS
    renderer, a code path the texture gradients share nothing with."""
    from oracle import render as R
    scene = sg.make_scene(0, n=24, T=4, seed=11)
    attrs = scene["texels"][:, 0, 0, :].astype(np.float64)
    scene["texels"] = np.broadcast_to(attrs[:, None, None, :], scene["texels"].shape).astype(np.float32).copy()
    attrs = scene["texels"][:, 0, 0, :].astype(np.float64)
    cam = sg.look_at_camera((3.0, 0.5, 0.8), 32, 32)
    env = sg.make_env(0, cube_res=8, irr_res=4, lut_res=16)
    dL = np.random.default_rng(21).normal(size=(32, 32, 4))
    gr = G.render_grads(scene, cam, env, dL)
    summed = gr["texels"].sum(axis=(1, 2))  # [n, 8]
    scale = np.abs(summed).max()
    assert scale > 0

    def S(a):
        return float((R.render_attributes_2dgs(scene, cam, env, a)["rgba"].numpy() * dL).sum())

    h = 1e-6
    for flat in np.argsort(-np.abs(summed).ravel())[:4]:
        k, c = np.unravel_index(flat, summed.shape)
        ap, am = attrs.copy(), attrs.copy()
        ap[k, c] += h
        am[k, c] -= h
        fd = (S(ap) - S(am)) / (2 * h)
        assert abs(fd - summed[k, c]) <= 1e-6 * scale + 1e-6 * abs(fd), (k, c, fd, summed[k, c])
