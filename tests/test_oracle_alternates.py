"""Pins of the oracle's admissible alternative results.

Where one discrete decision of a pixel (the support edge |u|, |v| <= 3, the
alpha >= 1/255 cut, the T < 1e-4 termination, the normal's orientation) lies
within FP32 error of its switching point, an FP32 renderer may take either
branch, and the oracle returns the result of the other branch beside the
definition's (render()["alt"]).  These tests build pixels that sit exactly at
such a point and check both results against closed forms of Eq. 2-3, and
that a pixel with two such decisions is masked instead.
"""
import numpy as np

import scenegen as sg
from oracle import render as R
from tests.helpers import cam_identity, fronto_scene

ALPHA_MAX = np.float64(np.float32(0.99))
ALPHA_MIN = np.float64(np.float32(1 / 255))
ATTR = np.array([0.6, 0.3, 0.2, 0.25, 0.5, 0.0, 0.0, 1.0], dtype=np.float32)


def env():
    return sg.constant_env(np.array([0.7, 0.5, 0.3], np.float32), lut=(0.625, 0.125))


def const_tex(n):
    return np.broadcast_to(ATTR, (n, 2, 2, 8)).copy()


def test_support_edge_gives_the_flipped_fragment():
    # pixel column 100 sees u = 3 + d (just outside) and column 99 sees it
    # just inside for a splat whose left edge is not in view: su = 1/8, the
    # centre x0 placed so that column 100's ray meets u = 3 + 2e-6
    su, sv, o = 0.125, 0.25, 0.9
    xr = (100.5 - 64.0) / 64.0
    x0 = np.float32(xr - su * (3.0 + 2e-6))
    sc = fronto_scene([[x0, 0.0, 1.0]], [[su, sv]], [o], const_tex(1))
    out = R.render(sc, cam_identity(), env())
    row = 64  # v = (64.5 - 64)/64 / sv, small
    v = (row + 0.5 - 64.0) / 64.0 / sv
    u = (xr - np.float64(x0)) / su
    assert 3.0 < u < 3.0 + 1e-5
    a_flip = np.float64(np.float32(o)) * np.exp(-(u * u + v * v) / 2.0)
    assert a_flip > ALPHA_MIN
    assert out["A"][row, 100].item() == 0.0           # the definition: outside the support
    assert bool(out["alt"]["mask"][row, 100])
    np.testing.assert_allclose(out["alt"]["A"][row, 100].item(), a_flip, rtol=1e-12)
    np.testing.assert_allclose(out["alt"]["T"][row, 100].item(), 1.0 - a_flip, rtol=1e-12)
    np.testing.assert_allclose(out["alt"]["X"][row, 100, :5].numpy(), a_flip * ATTR[:5].astype(np.float64),
                               rtol=1e-12)
    # the column next to it is far from the edge: a unique result
    assert not bool(out["alt"]["mask"][row, 98]) and not bool(out["ambiguous"][row, 98])
    assert out["A"][row, 98].item() > 0.0
    np.testing.assert_array_equal(out["alt"]["rgba"][row, 98].numpy(), out["rgba"][row, 98].numpy())
    # and on the inside of the edge the alternative drops the fragment
    x1 = np.float32(xr - su * (3.0 - 2e-6))
    out2 = R.render(fronto_scene([[x1, 0.0, 1.0]], [[su, sv]], [o], const_tex(1)), cam_identity(), env())
    assert out2["A"][row, 100].item() > 0.0 and bool(out2["alt"]["mask"][row, 100])
    assert out2["alt"]["A"][row, 100].item() == 0.0
    assert out2["alt"]["rgba"][row, 100].abs().max().item() == 0.0


def stacked(depths, opac):
    # fronto splats centred on the ray of pixel (63, 63): u = v = 0 there exactly
    means = [[-d / 128.0, -d / 128.0, d] for d in depths]
    return fronto_scene(means, [[0.1, 0.1]] * len(depths), opac, const_tex(len(depths)))


def test_termination_gives_one_more_fragment():
    # two layers at the 0.99 clamp leave T = (1 - 0.99f)^2 = 1e-4 (1 - 1.9e-6):
    # the definition stops there (T < 1e-4), the alternative blends the third
    out = R.render(stacked([1.0, 2.0, 3.0], [1.0, 1.0, 1.0]), cam_identity(), env())
    p = (63, 63)
    om = 1.0 - ALPHA_MAX
    A2 = ALPHA_MAX * (1.0 + om)
    A3 = A2 + ALPHA_MAX * om * om
    assert om * om < np.float64(np.float32(1e-4))
    np.testing.assert_allclose(out["A"][p].item(), A2, rtol=1e-14)
    np.testing.assert_allclose(out["T"][p].item(), om * om, rtol=1e-14)
    assert out["last"][p].item() == 1
    assert bool(out["alt"]["mask"][p]) and not bool(out["ambiguous"][p])
    np.testing.assert_allclose(out["alt"]["A"][p].item(), A3, rtol=1e-14)
    np.testing.assert_allclose(out["alt"]["T"][p].item(), om ** 3, rtol=1e-14)
    assert out["alt"]["last"][p].item() == 2
    # equal attributes in every layer: the colour scales with the coverage
    np.testing.assert_allclose(out["alt"]["rgba"][p][:3].numpy(), out["rgba"][p][:3].numpy() * (A3 / A2),
                               rtol=1e-12)


def test_termination_reached_just_above_threshold_stops_in_the_alternative():
    # a first layer of alpha a1 (the float32 just below the 0.99 clamp) so
    # that T after it and one clamped layer behind it sits just above 1e-4:
    # the definition goes on to the third layer, the alternative stops after
    # the second
    tmin = np.float64(np.float32(1e-4))
    om = 1.0 - ALPHA_MAX
    o1 = np.nextafter(np.float32(0.99), np.float32(0.0))  # the float32 just below the clamp
    a1 = np.float64(o1)
    t2 = (1.0 - a1) * om
    assert a1 < ALPHA_MAX and 0.0 < t2 / tmin - 1.0 < 2e-4
    out = R.render(stacked([1.0, 2.0, 3.0], [o1, 1.0, 1.0]), cam_identity(), env())
    p = (63, 63)
    assert out["last"][p].item() == 2 and bool(out["alt"]["mask"][p])
    assert out["alt"]["last"][p].item() == 1
    np.testing.assert_allclose(out["alt"]["T"][p].item(), t2, rtol=1e-12)
    np.testing.assert_allclose(out["T"][p].item(), t2 * om, rtol=1e-12)
    np.testing.assert_allclose(out["A"][p].item() - out["alt"]["A"][p].item(), ALPHA_MAX * t2, rtol=1e-9)


def test_two_decisions_near_their_thresholds_are_masked():
    # the termination of the clamped pair and, behind it, a splat whose alpha
    # equals the 1/255 cut: no unique pair of results, the pixel is masked
    out = R.render(stacked([1.0, 2.0, 3.0], [1.0, 1.0, np.float32(1 / 255)]), cam_identity(), env())
    p = (63, 63)
    assert bool(out["ambiguous"][p]) and not bool(out["alt"]["mask"][p])
    assert bool(out["grad_ambiguous"][p])
    # a few pixels away from the centre nothing is near a threshold
    q = (63, 70)
    assert not bool(out["ambiguous"][q]) and not bool(out["alt"]["mask"][q])
