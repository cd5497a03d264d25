"""Pins of the oracle's depth channel and normal-consistency loss (Sec. 3.6):
closed forms for planes, and central differences of L_n."""
import math

import numpy as np
import torch

import scenegen as sg
from oracle import loss as OL
from oracle import render as R
from tests.helpers import cam_identity, fronto_scene, twisted_quat


def plane_scene(phi, p=(0.0, 0.0, 2.0), s=0.6, o=0.99, nt=(0.0, 0.0, 1.0), T=4):
    """One large splat through p, rotated by phi about the y axis, with a
    constant texture whose tangent normal is nt."""
    tu = np.array([math.cos(phi), 0.0, -math.sin(phi)])
    tv = np.array([0.0, 1.0, 0.0])
    n = np.cross(tu, tv)
    q = twisted_quat(tu, tv, n)
    attr = np.array([0.5, 0.5, 0.5, 0.2, 0.5, *nt], dtype=np.float32)
    tex = np.broadcast_to(attr, (1, T, T, 8)).copy()
    sc = fronto_scene([list(p)], [[s, s]], [o], tex, quats=[q])
    # the normal of the stored (float32) quaternion, as the renderer sees it
    _, _, n_q = R.rotation_columns(torch.tensor(sc["quats"], dtype=torch.float64))
    return sc, n_q[0].numpy()


def test_depth_channel_is_coverage_times_hit_depth():
    for phi in (0.0, 0.5, -0.9):
        sc, n = plane_scene(phi)
        cam = cam_identity(W=64, H=64, f=40.0, cx=32.0, cy=32.0)
        out = R.render(sc, cam, sg.constant_env((0.5, 0.5, 0.5)))
        A, Z = out["A"].numpy(), out["Z"].numpy()
        xs = (np.arange(64) + 0.5 - 32.0) / 40.0
        d = np.stack(np.broadcast_arrays(xs[None, :], xs[:, None], np.ones((64, 64))), -1)
        tau = (np.array([0.0, 0.0, 2.0]) @ n) / (d @ n)  # ray-plane depth
        m = A > 0
        assert m.sum() > 200
        np.testing.assert_allclose(Z[m], A[m] * tau[m], rtol=1e-12)
        assert np.all(Z[~m] == 0.0)


def test_normal_loss_vanishes_on_a_plane_with_flat_normal_map():
    for phi in (0.0, 0.4, -0.7):
        sc, n = plane_scene(phi)
        cam = cam_identity(W=64, H=64, f=40.0, cx=32.0, cy=32.0)
        out = R.render(sc, cam, sg.constant_env((0.5, 0.5, 0.5)))
        L, mask, Nt = OL.depth_normal_loss(out["Z"], out["A"], out["X"], cam)
        assert mask.sum() > 100
        assert abs(float(L)) < 1e-12
        # the depth normal is the plane normal turned towards the camera
        facing = -n if n[2] > 0 else n
        np.testing.assert_allclose(Nt.numpy()[mask.numpy()], np.broadcast_to(facing, (int(mask.sum()), 3)),
                                   atol=1e-12)


def test_normal_loss_of_a_tilted_normal_map_is_one_minus_cos():
    theta = 0.3
    sc, n = plane_scene(0.25, nt=(math.sin(theta), 0.0, math.cos(theta)))
    cam = cam_identity(W=64, H=64, f=40.0, cx=32.0, cy=32.0)
    out = R.render(sc, cam, sg.constant_env((0.5, 0.5, 0.5)))
    L, mask, _ = OL.depth_normal_loss(out["Z"], out["A"], out["X"], cam)
    cnt = int(mask.sum())
    assert cnt > 100
    # tangent normal as stored (float32): cos = n_z / |n| in the splat frame
    nt = np.array([np.float32(math.sin(theta)), 0.0, np.float32(math.cos(theta))], dtype=np.float64)
    cos = nt[2] / np.linalg.norm(nt)
    np.testing.assert_allclose(float(L), cnt * (1.0 - cos) / (62 * 62), rtol=1e-10)


def test_normal_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(4)
    W = H = 24
    cam = cam_identity(W=W, H=H, f=20.0, cx=12.0, cy=12.0)
    Z = torch.tensor(rng.uniform(1.5, 2.5, size=(H, W)) * 0.9, dtype=torch.float64, requires_grad=True)
    A = torch.tensor(rng.uniform(0.8, 1.0, size=(H, W)), dtype=torch.float64, requires_grad=True)
    X = torch.tensor(rng.normal(size=(H, W, 8)), dtype=torch.float64, requires_grad=True)
    L, mask, _ = OL.depth_normal_loss(Z, A, X, cam)
    gZ, gA, gX = torch.autograd.grad(L, (Z, A, X))
    h = 1e-7
    for t, g, idx in ((Z, gZ, (5, 7)), (A, gA, (10, 3)), (X, gX, (8, 8, 6)), (Z, gZ, (1, 1))):
        with torch.no_grad():
            t[idx] += h
            lp = float(OL.depth_normal_loss(Z, A, X, cam)[0])
            t[idx] -= 2 * h
            lm = float(OL.depth_normal_loss(Z, A, X, cam)[0])
            t[idx] += h
        np.testing.assert_allclose(float(g[idx]), (lp - lm) / (2 * h), rtol=1e-5, atol=1e-10)
