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
