"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bar: tile/sort lists bit-exact; images within 1e-4 max-abs of an admissible
oracle result on every pixel: the definition's result, or, where exactly one
threshold decision of the pixel lies within FP32 error of flipping, the
result with that decision flipped.  Pixels with several such decisions are
masked, at most 0.1 % of them.
"""
import numpy as np
import pytest
import torch

import scenegen as sg
from oracle import keys as K
from oracle import render as R
from tests.helpers import admissible_errors, check_admissible

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4


@pytest.fixture(scope="module")
def P():
    import paper_2506_13348_b300 as P
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return P


def gpu_render(P, scene, env, cam, store="f32", env_store="f32"):
    sc = P.Scene.from_arrays(scene, env, store=store, env_store=env_store)
    out, saved = P.render(sc, cam, save=True)
    torch.cuda.synchronize()
    return sc, out, saved


def compare_lists(saved, kl, n):
    ids, rng, db = saved.lists(n)
    assert ids.size == kl["ids"].size
    np.testing.assert_array_equal(ids, kl["ids"])
    ref_rng = kl["tile_ranges"]
    nonempty = ref_rng[:, 1] > ref_rng[:, 0]
    np.testing.assert_array_equal(rng[nonempty], ref_rng[nonempty])
    assert np.all(rng[~nonempty, 1] == rng[~nonempty, 0])  # empty tiles are empty ranges
    vis = kl["view"]["visible"]
    np.testing.assert_array_equal(db[vis], kl["view"]["depth_bits"][vis])
    assert np.all(db[~vis] == 0xFFFFFFFF)


def compare_image(gpu_rgba, ref, tol=IMG_TOL, max_masked=1e-3, label=""):
    return check_admissible(gpu_rgba.detach().cpu().numpy(), ref, tol, max_masked, label)["max_err"]


def test_cfg0_keys_bit_exact_and_image(P):
    scene = sg.make_scene(0)
    env = sg.make_env(0)
    cam = sg.look_at_camera((4.0, 0.0, 0.0), 128, 128)
    kl = K.build_keys(scene, cam)
    sc, out, saved = gpu_render(P, scene, env, cam)
    compare_lists(saved, kl, len(scene["opacity"]))
    ref = R.render(scene, cam, env, keylist=kl)
    compare_image(out, ref, label="cfg0")
    # per-pixel forward state, against the same admissible results
    g, tr, last = saved.pixels(0)
    amb = ref["ambiguous"].numpy()
    assert admissible_errors(g.cpu().numpy(), ref, "X")[~amb].max() <= IMG_TOL
    assert admissible_errors(tr.cpu().numpy(), ref, "T")[~amb].max() <= IMG_TOL
    # last blended fragment: oracle index is within the tile list
    tiles_x = kl["view"]["tiles_x"]
    yy, xx = np.meshgrid(np.arange(128), np.arange(128), indexing="ij")
    start = kl["tile_ranges"][(yy // 16) * tiles_x + xx // 16, 0]
    gl = last.cpu().numpy()
    ok = np.zeros_like(amb)
    for ol in (ref["last"].numpy(), ref["alt"]["last"].numpy()):
        ok |= gl == np.where(ol >= 0, start + ol, -1)
    assert (ok | amb).all()


@pytest.mark.parametrize("seed,W,H,eye", [(3, 100, 77, (2.5, 1.5, 1.0)), (5, 64, 48, (0.0, -3.0, 2.0)),
                                          (8, 33, 129, (1.2, 1.2, -1.8))])
def test_small_scenes_ragged_sizes(P, seed, W, H, eye):
    scene = sg.make_scene(1, n=600, T=4, seed=seed)
    env = sg.make_env(seed, cube_res=16, levels=3, irr_res=8, lut_res=32)
    cam = sg.look_at_camera(eye, W, H)
    kl = K.build_keys(scene, cam)
    sc, out, saved = gpu_render(P, scene, env, cam)
    compare_lists(saved, kl, 600)
    compare_image(out, R.render(scene, cam, env, keylist=kl), label=f"ragged {W}x{H}")


def test_empty_and_culled_scenes(P):
    env = sg.make_env(0, cube_res=8, irr_res=4, lut_res=16)
    cam = sg.look_at_camera((4.0, 0.0, 0.0), 40, 24)
    empty = dict(means=np.zeros((0, 3), np.float32), quats=np.zeros((0, 4), np.float32),
                 scales=np.zeros((0, 2), np.float32), opacity=np.zeros(0, np.float32),
                 texels=np.zeros((0, 4, 4, 8), np.float32), T=4)
    sc, out, saved = gpu_render(P, empty, env, cam)
    assert torch.count_nonzero(out).item() == 0
    assert saved.sizes()[0] == 0
    # every splat behind the camera: nothing binned
    scene = sg.make_scene(0, n=50, T=2, seed=1)
    scene["means"][:, 0] += 10.0
    sc, out, saved = gpu_render(P, scene, env, cam)
    assert saved.sizes()[0] == 0
    assert torch.count_nonzero(out).item() == 0


def test_forward_deterministic_and_batched_equals_alone(P):
    scene = sg.make_scene(1, n=3000, T=4, seed=2)
    env = sg.make_env(2, cube_res=16, levels=2, irr_res=8, lut_res=32)
    cams = [sg.look_at_camera(e, w, h) for e, w, h in [((3.0, 0.5, 0.5), 96, 64), ((0.5, 3.5, 0.2), 50, 70),
                                                        ((-2.0, -2.0, 2.0), 128, 128)]]
    sc = P.Scene.from_arrays(scene, env)
    alone = [P.render(sc, c)[0].clone() for c in cams]
    again = [P.render(sc, c)[0].clone() for c in cams]
    outs, _ = P.render_views([sc] * 3, cams)
    torch.cuda.synchronize()
    for a, b, c in zip(alone, again, outs):
        assert torch.equal(a, b)
        assert torch.equal(a, c)


@pytest.mark.parametrize("store", ["bf16", "f16"])
def test_reduced_precision_atlas_pipeline_parity(P, store):
    # the oracle is fed the same rounded texels: pipeline parity within 1e-4
    scene = sg.make_scene(0, n=400, T=8, seed=4)
    env = sg.make_env(4, cube_res=16, irr_res=8, lut_res=32)
    cam = sg.look_at_camera((3.0, 1.0, 0.5), 96, 96)
    tt = torch.from_numpy(scene["texels"])
    rounded = tt.to(torch.bfloat16 if store == "bf16" else torch.float16).float().numpy()
    sc, out, saved = gpu_render(P, scene, env, cam, store=store)
    ref = R.render(dict(scene, texels=rounded), cam, env)
    compare_image(out, ref, label=f"{store} atlas")


def test_fragment_counts_match_oracle(P):
    """The counting pass behind the bench's FLOP model (E evaluated, C blended
    fragments) counts what the oracle's definition counts."""
    scene = sg.make_scene(0)
    env = sg.make_env(0)
    cam = sg.look_at_camera((4.0, 0.0, 0.0), 128, 128)
    kl = K.build_keys(scene, cam)
    sc, out, saved = gpu_render(P, scene, env, cam)
    st = saved.frag_stats()
    ref = R.render(scene, cam, env, keylist=kl)
    # pixels with a decision near its switching point may count differently
    amb = ref["ambiguous"].numpy() | ref["alt"]["mask"].numpy()
    tiles_x = kl["view"]["tiles_x"]
    yy, xx = np.meshgrid(np.arange(128), np.arange(128), indexing="ij")
    rng = kl["tile_ranges"][(yy // 16) * tiles_x + xx // 16]
    list_len = rng[..., 1] - rng[..., 0]
    slack = int(list_len[amb].sum())
    e_ref = int(ref["n_eval"].sum())
    c_ref = int(ref["n_contrib"].sum())
    assert st["n_pairs"] == kl["ids"].size
    assert st["n_visible"] == int(kl["view"]["visible"].sum())
    assert e_ref > 1000 and c_ref > 1000
    assert abs(st["n_evaluated"] - e_ref) <= slack, (st, e_ref, slack)
    assert abs(st["n_blended"] - c_ref) <= slack, (st, c_ref, slack)
    e_ok = int(ref["n_eval"].numpy()[~amb].sum())
    assert e_ok <= st["n_evaluated"] <= e_ok + slack


def oracle_texels_read(scene, cam, kl, cell_band=1e-4):
    """Sets of (splat, texel) pairs the definition's blended fragments read
    (each reads the four clamped bilinear corners of Eq. 6): 'sure' from
    unmasked pixels and fragments clear of a bilinear cell boundary, 'maybe'
    adding the corners of both sides of a near-boundary floor and of every
    fragment in reach of a masked pixel; and the splats blended likewise."""
    params = R.to_params(scene)
    T = params["texels"].shape[1]
    W, H = int(cam["W"]), int(cam["H"])
    tiles_x, tiles_y = kl["view"]["tiles_x"], kl["view"]["tiles_y"]
    sure, maybe, items_sure, items_maybe = set(), set(), set(), set()

    def corners(sid, x, y):
        out = []
        for i0 in {int(np.floor(x - cell_band)), int(np.floor(x)), int(np.floor(x + cell_band))}:
            for j0 in {int(np.floor(y - cell_band)), int(np.floor(y)), int(np.floor(y + cell_band))}:
                for jj in (max(j0, 0), min(j0 + 1, T - 1)):
                    for ii in (max(i0, 0), min(i0 + 1, T - 1)):
                        out.append((sid, jj * T + ii))
        return out

    for tl in range(tiles_x * tiles_y):
        c = R.tile_candidates(kl, tl)
        if c.size == 0:
            continue
        tx, ty = tl % tiles_x, tl // tiles_x
        xs = np.arange(tx * K.TILE, min(W, (tx + 1) * K.TILE))
        ys = np.arange(ty * K.TILE, min(H, (ty + 1) * K.TILE))
        gy, gx = np.meshgrid(ys, xs, indexing="ij")
        cand = torch.from_numpy(np.ascontiguousarray(np.broadcast_to(c, (gx.size, c.size))).astype(np.int64))
        fr = R.fragments(params, cam, gx.ravel(), gy.ravel(), cand, R.DEFAULT_MARGINS)
        masked = (fr["ambiguous"] | fr["alt_mask"]).numpy()
        bl = fr["blended"].numpy()
        u, v = fr["u"].numpy(), fr["v"].numpy()
        reach = (np.abs(u) <= 3.001) & (np.abs(v) <= 3.001)
        xt = (u + 3.0) / 6.0 * T - 0.5
        yt = (v + 3.0) / 6.0 * T - 0.5
        cn = cand.numpy()
        for p_, l_ in zip(*np.nonzero(bl | (masked[:, None] & reach))):
            sid = int(cn[p_, l_])
            cs = corners(sid, xt[p_, l_], yt[p_, l_])
            maybe.update(cs)
            items_maybe.add(sid)
            if bl[p_, l_] and not masked[p_]:
                items_sure.add(sid)
                fx, fy = xt[p_, l_] - np.floor(xt[p_, l_]), yt[p_, l_] - np.floor(yt[p_, l_])
                if min(fx, 1 - fx, fy, 1 - fy) > cell_band:
                    sure.update(cs)
    return sure, maybe, items_sure, items_maybe


def test_texels_read_match_oracle(P):
    """The statistics pass's distinct texels read by blended fragments (the
    algorithmic texel bytes of the bench's traffic ratio) and distinct
    splats blended lie between what the definition certainly reads and what
    an admissible FP32 evaluation may read."""
    scene = sg.make_scene(0)
    env = sg.make_env(0)
    cam = sg.look_at_camera((4.0, 0.0, 0.0), 128, 128)
    kl = K.build_keys(scene, cam)
    sc, out, saved = gpu_render(P, scene, env, cam)
    st = saved.frag_stats()
    sure, maybe, items_sure, items_maybe = oracle_texels_read(scene, cam, kl)
    print(f"[texels] gpu {st['n_texels_read']} oracle sure {len(sure)} maybe {len(maybe)}; "
          f"items gpu {st['n_items_blended']} sure {len(items_sure)} maybe {len(items_maybe)}")
    assert len(sure) > 1000
    assert len(sure) <= st["n_texels_read"] <= len(maybe)
    assert len(items_sure) <= st["n_items_blended"] <= len(items_maybe)
    assert st["n_items_blended"] <= st["n_visible"]


def test_fp32_rate_probe(P):
    """The measured FP32 FMA rate (roofline denominator) is plausible for one
    B300-class GPU: 128 FP32 lanes x 148 SMs x ~2 GHz ~ 77 TFLOP/s."""
    from paper_2506_13348_b300 import _lib
    scalar, paired = _lib.measure_fp32_peak(0)
    assert 20.0 < scalar < 120.0, scalar
    assert 20.0 < paired < 240.0, paired


def test_pair_count_past_32_bits_is_a_capacity_error(P):
    """300k splats that each cover every tile of a 2048^2 view: 4.9e9
    (tile, splat) pairs, past what the 32-bit count scan can hold.  The
    64-bit total catches it before any pair buffer is sized from the
    wrapped scan: TS_ERR_CAPACITY, and the scene still renders afterwards
    with a camera that sees a few splats."""
    n = 300_000
    rng = np.random.default_rng(1)
    means = np.zeros((n, 3), np.float32)
    means[:, 2] = 5.0 + rng.uniform(0, 1, n).astype(np.float32)
    scene = dict(means=means, quats=np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
                 scales=np.full((n, 2), 10.0, np.float32), opacity=np.full(n, 0.5, np.float32),
                 texels=np.full((n, 1, 1, 8), 0.5, np.float32), T=1)
    env = sg.make_env(0, cube_res=8, irr_res=4, lut_res=16)
    cam = dict(R=np.eye(3, dtype=np.float32), t=np.zeros(3, np.float32), fx=np.float32(1024.0),
               fy=np.float32(1024.0), cx=np.float32(1024.0), cy=np.float32(1024.0), W=2048, H=2048)
    sc = P.Scene.from_arrays(scene, env)
    with pytest.raises(P.TexSplatError, match="CAPACITY"):
        P.render(sc, cam)
    small = dict(cam, W=64, H=64, cx=np.float32(32.0), cy=np.float32(32.0), fx=np.float32(32.0),
                 fy=np.float32(32.0))
    # 16 tiles x 300k splats = 4.8e6 pairs: renders
    out, _ = P.render(sc, small)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all() and out[..., 3].min().item() > 0.99


@pytest.mark.parametrize("n", [1, 1023, 1025, (1 << 18) + 1])
def test_depth_sort_block_and_path_boundaries(P, n):
    """Key lists bit-exact at splat counts around the sort's block size
    (1024 keys) and just past the small-sort limit (2^18 keys: the 64-bit
    depth sort switches to 2048-key blocks), with ragged last blocks."""
    scene = sg.make_scene(0, n=n, T=2, seed=n % 97)
    env = sg.make_env(0, cube_res=8, irr_res=4, lut_res=16)
    cam = sg.look_at_camera((3.5, 0.4, 0.3), 96, 80)
    kl = K.build_keys(scene, cam)
    sc, out, saved = gpu_render(P, scene, env, cam)
    compare_lists(saved, kl, n)
