"""Pins of the FP64 shading and cube/LUT sampling (oracle/shading.py)."""
import math

import numpy as np
import torch

import scenegen as sg
from oracle import shading as S


def t64(a):
    return torch.tensor(np.asarray(a, dtype=np.float64))


def test_cube_face_coords_textbook_cases():
    # OpenGL cube-map face selection table: major axis picks the face; (s,t)
    # from (sc/|ma| + 1)/2, (tc/|ma| + 1)/2
    cases = {
        (1.0, 0.0, 0.0): (0, 0.5, 0.5),
        (-1.0, 0.0, 0.0): (1, 0.5, 0.5),
        (0.0, 1.0, 0.0): (2, 0.5, 0.5),
        (0.0, -1.0, 0.0): (3, 0.5, 0.5),
        (0.0, 0.0, 1.0): (4, 0.5, 0.5),
        (0.0, 0.0, -1.0): (5, 0.5, 0.5),
        (1.0, -0.5, 0.25): (0, 0.375, 0.75),   # +x: sc = -z, tc = -y
        (-1.0, 0.5, 0.25): (1, 0.625, 0.25),   # -x: sc = z, tc = -y
        (0.5, 1.0, -0.25): (2, 0.75, 0.375),   # +y: sc = x, tc = z
        (0.5, -1.0, -0.25): (3, 0.75, 0.625),  # -y: sc = x, tc = -z
        (0.5, 0.25, 1.0): (4, 0.75, 0.375),    # +z: sc = x, tc = -y
        (0.5, 0.25, -1.0): (5, 0.25, 0.375),   # -z: sc = -x, tc = -y
    }
    for d, (f, s, t) in cases.items():
        face, ss, tt, _ = S.cube_face_coords(t64([d]))
        assert int(face[0]) == f, d
        assert abs(float(ss[0]) - s) < 1e-15 and abs(float(tt[0]) - t) < 1e-15, d


def test_cube_texel_centres_round_trip():
    # directions through texel centres (generator) map back to those texels
    R = 8
    d = sg.scenes.cube_texel_dirs(R).reshape(-1, 3)
    face, s, t, _ = S.cube_face_coords(t64(d))
    fi = np.repeat(np.arange(6), R * R)
    jj, ii = np.meshgrid(np.arange(R), np.arange(R), indexing="ij")
    np.testing.assert_array_equal(face.numpy(), fi)
    np.testing.assert_allclose(s.numpy() * R - 0.5, np.tile(ii.ravel(), 6), atol=1e-12)
    np.testing.assert_allclose(t.numpy() * R - 0.5, np.tile(jj.ravel(), 6), atol=1e-12)
    # so sampling a cube at its texel directions returns the texels
    cube = np.random.default_rng(0).uniform(size=(6, R, R, 3))
    got = S.cube_sample(t64(cube), t64(d)).numpy()
    np.testing.assert_allclose(got, cube.reshape(-1, 3), atol=1e-12)


def test_irradiance_cube_matches_analytic_sh():
    # the irradiance cube holds the SH cosine convolution at texel centres;
    # bilinear lookups between centres approximate the smooth function
    env = sg.make_env(3, cube_res=8, irr_res=32, lut_res=8)
    rng = np.random.default_rng(1)
    d = rng.normal(size=(2000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    got = S.cube_sample(t64(env["irr"]), t64(d)).numpy()
    ref = sg.scenes.sh_irradiance(env["sh"], d)
    assert np.abs(got - ref).max() < 2e-2 * np.abs(ref).max()
    # constant radiance c: irradiance pi * c
    y00 = sg.scenes._real_sh(0, np.array([[0, 0, 1.0]]))[0, 0]
    coeffs = np.zeros((25, 3))
    coeffs[0] = 0.5 / y00  # radiance 0.5 everywhere
    np.testing.assert_allclose(sg.scenes.sh_irradiance(coeffs, d), math.pi * 0.5, rtol=1e-12)


def test_lut_texel_centres_and_bilinear():
    lut = np.random.default_rng(2).uniform(size=(8, 8, 2))
    nv = (np.arange(8) + 0.5) / 8
    got = S.lut_sample(t64(lut), t64(np.tile(nv, 8)), t64(np.repeat(nv, 8))).numpy()
    np.testing.assert_allclose(got, lut.reshape(-1, 2), atol=1e-14)
    # midway between two NdotV texel centres: the average
    mid = S.lut_sample(t64(lut), t64([1.0 / 8]), t64([0.5 / 8])).numpy()[0]
    np.testing.assert_allclose(mid, 0.5 * (lut[0, 0] + lut[0, 1]), atol=1e-14)


def test_constant_environment_closed_form():
    # constant radiance c everywhere, LUT constant (A0, B0): colour =
    # A [Lam (1-M) c + (F0 A0 + B0) c]; independent of normal and view (Eq. 10-12)
    c = np.array([0.4, 0.9, 0.2])
    A0, B0 = 0.75, 0.0625
    env = sg.constant_env(c, cube_res=4, levels=3, irr_res=2, lut=(A0, B0))
    envt = dict(spec=[t64(m) for m in env["spec"]], irr=t64(env["irr"]), lut=t64(env["lut"]))
    rng = np.random.default_rng(4)
    P = 500
    A = rng.uniform(0.05, 1.0, size=P)
    lam = rng.uniform(size=(P, 3))
    met = rng.uniform(size=P)
    rough = rng.uniform(0.05, 1, size=P)
    N = rng.normal(size=(P, 3))
    X = np.concatenate([lam * A[:, None], (met * A)[:, None], (rough * A)[:, None], N], 1)
    d = rng.normal(size=(P, 3))
    col = S.shade(t64(X), t64(A), t64(d), envt).numpy()
    f0 = 0.04 * (1 - met[:, None]) + lam * met[:, None]
    cf = np.float32(c).astype(np.float64)
    ref = A[:, None] * (lam * (1 - met[:, None]) * cf + (f0 * A0 + B0) * cf)
    np.testing.assert_allclose(col[:, :3], ref, atol=1e-6)
    np.testing.assert_allclose(col[:, 3], A, atol=0)


def test_reflection_direction_and_lod_selection():
    # a mirror-like pixel (roughness 0) facing the camera head-on reflects the
    # view ray straight back: w_r = w_o; with a two-level cube whose levels are
    # constant 1 and 3, roughness r selects 1 + 2r (linear between levels)
    levels = [np.full((6, 4, 4, 3), 1.0), np.full((6, 2, 2, 3), 3.0)]
    lut = np.zeros((4, 4, 2))
    lut[..., 1] = 1.0  # L_s = spec
    env = dict(spec=[t64(m) for m in levels], irr=t64(np.zeros((6, 2, 2, 3))), lut=t64(lut))
    for r in [0.0, 0.25, 0.5, 1.0]:
        X = np.array([[0.0, 0.0, 0.0, 0.0, r, 0.0, 0.0, -1.0]])
        col = S.shade(t64(X), t64([1.0]), t64([[0.0, 0.0, 1.0]]), env).numpy()
        np.testing.assert_allclose(col[0, :3], 1.0 + 2.0 * r, atol=1e-12)
    # w_r = 2 (N.w_o) N - w_o for a tilted normal: sample a cube that is 1 on
    # the +x face only
    cube = np.zeros((6, 4, 4, 3))
    cube[0] = 1.0
    env1 = dict(spec=[t64(cube)], irr=t64(np.zeros((6, 2, 2, 3))), lut=t64(lut))
    n = np.array([np.sin(np.pi / 8), 0.0, -np.cos(np.pi / 8)])  # 22.5 deg towards +x
    X = np.concatenate([[0, 0, 0, 0, 0.0], n])[None]
    col = S.shade(t64(X), t64([1.0]), t64([[0.0, 0.0, 1.0]]), env1).numpy()
    # w_o = (0,0,-1), w_r is 45 deg between -z and +x: on the +x/-z face edge,
    # ties go to x -> +x face
    assert col[0, 0] == 1.0
