"""Failure detection without a GPU fault: the radix sort's inter-block wait
is bounded; a pass whose predecessor never runs reports TS_ERR_TIMEOUT
through the host, and the device stays usable."""
import time

import numpy as np

import pytest
import torch

import scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2506_13348_b300 as P
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return P


def test_sort_wait_runs_out_and_is_reported(P):
    from paper_2506_13348_b300 import _lib
    t0 = time.time()
    st = _lib.lib().ts_selftest_sort_wait(0, None)
    dt = time.time() - t0
    assert _lib.STATUS[st] == "TS_ERR_TIMEOUT", _lib.lib().ts_last_error()
    assert dt < 30.0
    # the flag was cleared and the context is usable: a render goes through
    scene = sg.make_scene(0, n=256, T=4, seed=0)
    env = sg.make_env(0, cube_res=8, irr_res=4, lut_res=16)
    sc = P.Scene.from_arrays(scene, env)
    out, _ = P.render(sc, sg.look_at_camera((4.0, 0.0, 0.0), 64, 64))
    torch.cuda.synchronize()
    assert torch.isfinite(out).all() and out[..., 3].max().item() > 0.5


def _bad(scene, key, idx, value):
    out = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
    out[key][idx] = value
    return out


@pytest.mark.parametrize("key,idx,value,reason", [
    ("means", (7, 1), np.nan, b"centre"),
    ("means", (3, 0), np.inf, b"centre"),
    ("quats", 11, 0.0, b"quaternion"),
    ("scales", (5, 0), 0.0, b"scale"),
    ("scales", (9, 1), -0.1, b"scale"),
    ("opacity", 2, 1.5, b"opacity"),
    ("opacity", 4, np.nan, b"opacity"),
])
def test_malformed_upload_is_rejected_and_scene_kept(P, key, idx, value, reason):
    """A malformed geometry upload returns TS_ERR_ARG naming the first bad
    splat and the reason, and leaves the previous geometry in place: the
    scene renders bit-identically afterwards."""
    from paper_2506_13348_b300 import _lib
    scene = sg.make_scene(0, n=256, T=4, seed=0)
    env = sg.make_env(0, cube_res=8, irr_res=4, lut_res=16)
    cam = sg.look_at_camera((4.0, 0.0, 0.0), 64, 64)
    sc = P.Scene.from_arrays(scene, env)
    before, _ = P.render(sc, cam)
    before = before.clone()
    bad = _bad(scene, key, idx, value)
    with pytest.raises(P.TexSplatError, match="TS_ERR_ARG"):
        sc.upload_gaussians(bad["means"], bad["quats"], bad["scales"], bad["opacity"])
    msg = _lib.lib().ts_last_error()
    assert reason in msg and b"first index" in msg, msg
    first = idx[0] if isinstance(idx, tuple) else idx
    assert f"first index {first}".encode() in msg, msg
    after, _ = P.render(sc, cam)
    torch.cuda.synchronize()
    assert torch.equal(before, after)


def test_injected_allocation_failures_leave_state_intact(P):
    """Allocation failures injected on the host (the k-th library allocation
    fails as out-of-memory) at every allocation of a geometry upload, an
    atlas upload, an environment upload and a render: each call returns
    TS_ERR_OOM, the scene keeps what it had, and the next render equals the
    first bit for bit."""
    from paper_2506_13348_b300 import _lib
    L = _lib.lib()
    scene = sg.make_scene(0, n=300, T=4, seed=3)
    env = sg.make_env(0, cube_res=8, levels=2, irr_res=4, lut_res=16)
    cam = sg.look_at_camera((3.5, 0.5, 0.5), 64, 48)
    sc = P.Scene.from_arrays(scene, env)
    ref, _ = P.render(sc, cam)
    ref = ref.clone()
    other = sg.make_scene(0, n=300, T=4, seed=4)
    calls = [
        ("geometry", lambda: sc.upload_gaussians(other["means"], other["quats"], other["scales"], other["opacity"])),
        ("atlas", lambda: sc.upload_atlas(other["texels"], "bf16")),
        ("envmap", lambda: sc.upload_envmap(sg.make_env(5, cube_res=8, levels=2, irr_res=4, lut_res=16), "f16")),
        ("render", lambda: P.render(sc, cam, save=True)),
    ]
    try:
        for name, fn in calls:
            failures = 0
            for k in range(64):
                assert L.ts_debug_fail_alloc(k) == 0
                try:
                    fn()
                except P.TexSplatError as e:
                    assert "TS_ERR_OOM" in str(e), (name, k, str(e))
                    failures += 1
                    out, _ = P.render(sc, cam)
                    torch.cuda.synchronize()
                    assert torch.equal(out, ref), (name, k)
                    continue
                # the call made fewer than k+1 allocations: every one was tried
                L.ts_debug_fail_alloc(-1)
                break
            assert failures >= 1, name
            if name != "render":  # a successful upload changed the scene: restore it
                L.ts_debug_fail_alloc(-1)
                sc.upload_gaussians(scene["means"], scene["quats"], scene["scales"], scene["opacity"])
                sc.upload_atlas(scene["texels"], "f32")
                sc.upload_envmap(env, "f32")
                out, _ = P.render(sc, cam)
                torch.cuda.synchronize()
                assert torch.equal(out, ref), name
    finally:
        L.ts_debug_fail_alloc(-1)


def test_backward_after_a_reupload_is_refused(P):
    """A saved forward keeps pointers into its scene's buffers; after an
    upload replaced them (new texels, geometry or environment), the backward
    and the fragment recount return TS_ERR_STATE instead of reading freed
    memory, and a fresh render's backward works again."""
    scene = sg.make_scene(0, n=300, T=4, seed=3)
    env = sg.make_env(0, cube_res=8, levels=1, irr_res=4, lut_res=16)
    cam = sg.look_at_camera((3.5, 0.5, 0.5), 64, 48)
    sc = P.Scene.from_arrays(scene, env)
    dl = torch.ones(48, 64, 4, device="cuda")
    for redo in (lambda: sc.upload_atlas(scene["texels"], "f32"),
                 lambda: sc.upload_gaussians(scene["means"], scene["quats"], scene["scales"], scene["opacity"]),
                 lambda: sc.upload_envmap(env, "f32")):
        _, saved = P.render(sc, cam, save=True)
        redo()
        with pytest.raises(P.TexSplatError, match="TS_ERR_STATE"):
            P.render_backward(saved, dl, P.zero_grads(sc))
        with pytest.raises(P.TexSplatError, match="TS_ERR_STATE"):
            saved.frag_stats()
        saved.release()
        _, saved = P.render(sc, cam, save=True)
        g = P.zero_grads(sc)
        P.render_backward(saved, dl, g)
        torch.cuda.synchronize()
        assert float(g["texels"].abs().sum()) > 0.0
        saved.release()


def test_server_budget_limits(P):
    """A zero-byte arena is refused at creation; a request larger than the
    arena is rejected at submission (TS_ERR_CAPACITY, counted), and a
    request that fits is still served."""
    from paper_2506_13348_b300 import _lib
    import ctypes as C
    h = C.c_void_p()
    assert _lib.STATUS[_lib.lib().ts_server_create(C.byref(h), 0, 0, 1, 1)] == "TS_ERR_ARG"
    scene = sg.make_scene(0, n=256, T=4, seed=0)
    env = sg.make_env(0, cube_res=8, irr_res=4, lut_res=16)
    sc = P.Scene.from_arrays(scene, env)
    small = sg.look_at_camera((4.0, 0.0, 0.0), 32, 32)
    big = sg.look_at_camera((4.0, 0.0, 0.0), 2048, 2048)
    srv = P.Server(device=0, arena_bytes=64 << 20, n_streams=1, max_batch=2)
    try:
        with pytest.raises(P.TexSplatError, match="CAPACITY"):
            srv.submit(sc, big)
        t = srv.submit(sc, small)
        img = torch.empty(32, 32, 4, dtype=torch.float32, device="cuda")
        srv.wait(t, img)
        ref, _ = P.render(sc, small)
        torch.cuda.synchronize()
        assert torch.equal(img, ref)
        assert srv.stats()["rejected"] == 1
    finally:
        srv.close()
