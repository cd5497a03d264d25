"""ts_render_noalloc: the render entry point that allocates no device memory.

It exists for callers that cannot allocate while they render (a renderer
inside a host application that owns the device budget, a real-time frame
loop, a plugin limited to the buffers it is given).  This file is collected
last on purpose.  It calls the entry point through the C ABI on two views in
a row (the second call, on fewer splats, runs on the working set the first
one left behind) and checks each image against the allocating entry point,
ts_render, bit for bit (the same kernels run), and that the calls allocate
nothing; then the limits.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import scenegen as sg

pytestmark = pytest.mark.gpu


def _call(L, arrs, env, cam, out, stream):
    import paper_2506_13348_b300 as P
    means, quats, scales, opac, tex, spec, irr, lut = arrs
    c = P.make_camera(cam)
    return L.ts_render_noalloc(means.shape[0], means.data_ptr(), quats.data_ptr(), scales.data_ptr(),
                               opac.data_ptr(), tex.shape[1], tex.data_ptr(), len(env["spec"]),
                               env["spec"][0].shape[1], spec.data_ptr(), irr.shape[1], irr.data_ptr(),
                               lut.shape[0], lut.data_ptr(), C.byref(c), out.data_ptr(),
                               C.c_void_p(stream.cuda_stream))


def _device_arrays(scene, env, dev):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)  # noqa: E731
    spec = torch.cat([t(m).reshape(-1) for m in env["spec"]])
    return [t(scene[k]) for k in ("means", "quats", "scales", "opacity", "texels")] + [spec, t(env["irr"]),
                                                                                        t(env["lut"])]


def test_noalloc_render_matches_ts_render_twice():
    """Two calls in a row, the second on fewer splats than the first (stale
    ids and keys of the first call lie beyond the second's count in the
    shared array): each image equals ts_render's bit for bit (same kernels),
    and the calls allocate nothing (device free memory and torch's pool
    unchanged across them)."""
    import paper_2506_13348_b300 as P
    from paper_2506_13348_b300 import _lib

    L = _lib.lib()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    env = sg.make_env(12, cube_res=16, levels=3, irr_res=8, lut_res=32)
    cases = [(sg.make_scene(1, n=3000, T=4, seed=12), sg.look_at_camera((2.6, 1.2, 0.9), 160, 120)),
             (sg.make_scene(1, n=1200, T=4, seed=13), sg.look_at_camera((-1.5, 2.5, -1.0), 72, 96))]
    stream = torch.cuda.current_stream()
    prepared = []
    for scene, cam in cases:
        ref, _ = P.render(P.Scene.from_arrays(scene, env), cam)
        out = torch.full((cam["H"], cam["W"], 4), float("nan"), dtype=torch.float32, device=dev)
        prepared.append((_device_arrays(scene, env, dev), cam, ref, out))
    _call(L, prepared[0][0], env, prepared[0][1], prepared[0][3], stream)  # the first call's set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    pool0 = torch.cuda.memory_stats(dev).get("allocation.all.allocated", 0)
    for arrs, cam, ref, out in prepared:
        out.fill_(float("nan"))
    status = [_call(L, arrs, env, cam, out, stream) for arrs, cam, ref, out in prepared]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0
    assert torch.cuda.memory_stats(dev).get("allocation.all.allocated", 0) == pool0
    for st, (arrs, cam, ref, out) in zip(status, prepared):
        assert st == 0, L.ts_last_error()
        assert (out[..., 3] > 0).sum() > 100
        assert torch.equal(out, ref), (out - ref).abs().max().item()


def test_noalloc_pair_limit_after_binning_then_renders_again():
    """2000 splats that each cover every tile of a 1920x1080 view: 16 M
    (tile, splat) pairs, past the fixed 2^20; the limit is found after
    binning (TS_ERR_CAPACITY), and the next call renders normally."""
    import paper_2506_13348_b300 as P
    from paper_2506_13348_b300 import _lib

    L = _lib.lib()
    dev = torch.device("cuda", 0)
    env = sg.make_env(0, cube_res=8, irr_res=4, lut_res=16)
    n = 2000
    big = dict(means=np.tile(np.array([0.0, 0.0, 5.0], np.float32), (n, 1)),
               quats=np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
               scales=np.full((n, 2), 10.0, np.float32), opacity=np.full(n, 0.5, np.float32),
               texels=np.full((n, 1, 1, 8), 0.5, np.float32), T=1)
    big["means"][:, 2] += np.linspace(0.0, 1.0, n, dtype=np.float32)
    cam = dict(R=np.eye(3, dtype=np.float32), t=np.zeros(3, np.float32), fx=np.float32(1000.0),
               fy=np.float32(1000.0), cx=np.float32(960.0), cy=np.float32(540.0), W=1920, H=1080)
    stream = torch.cuda.current_stream()
    out = torch.zeros(1080, 1920, 4, dtype=torch.float32, device=dev)
    st = _call(L, _device_arrays(big, env, dev), env, cam, out, stream)
    assert _lib.STATUS[st] == "TS_ERR_CAPACITY", L.ts_last_error()
    assert b"pairs" in L.ts_last_error()
    scene = sg.make_scene(1, n=800, T=4, seed=14)
    cam2 = sg.look_at_camera((2.0, -2.0, 1.0), 64, 48)
    ref, _ = P.render(P.Scene.from_arrays(scene, env), cam2)
    out2 = torch.full((48, 64, 4), float("nan"), dtype=torch.float32, device=dev)
    st = _call(L, _device_arrays(scene, env, dev), env, cam2, out2, stream)
    assert st == 0, L.ts_last_error()
    torch.cuda.synchronize()
    assert torch.equal(out2, ref)


def test_noalloc_rejects_sizes_beyond_its_limits():
    from paper_2506_13348_b300 import _lib
    import paper_2506_13348_b300 as P

    L = _lib.lib()
    c = P.make_camera(sg.look_at_camera((4.0, 0.0, 0.0), 4096, 4096))  # 65536 tiles > 8192
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    p = dummy.data_ptr()
    assert L.ts_render_noalloc(1 << 20, p, p, p, p, 4, p, 1, 8, p, 4, p, 8, p, C.byref(c), p, None) == 3
    assert L.ts_render_noalloc(10, p, p, p, p, 4, p, 1, 8, p, 4, p, 8, p, C.byref(c), p, None) == 3
    assert b"tiles" in L.ts_last_error()
