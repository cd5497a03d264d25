"""ts_render_noalloc: the render entry point that allocates no device memory.

It exists for callers that cannot allocate while they render (a renderer
inside a host application that owns the device budget, a real-time frame
loop, a plugin limited to the buffers it is given).  This file is collected
last on purpose.  It calls the entry point through the C ABI on two views in
a row (the second call runs on the working set the first one left behind)
and checks each image against the allocating entry point, ts_render, within
the image tolerance of the other parity tests.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import scenegen as sg

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4


def test_noalloc_render_matches_ts_render_twice():
    import paper_2506_13348_b300 as P
    from paper_2506_13348_b300 import _lib

    L = _lib.lib()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    scene = sg.make_scene(1, n=3000, T=4, seed=12)
    env = sg.make_env(12, cube_res=16, levels=3, irr_res=8, lut_res=32)
    cams = [sg.look_at_camera((2.6, 1.2, 0.9), 160, 120), sg.look_at_camera((-1.5, 2.5, -1.0), 72, 96)]

    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)  # noqa: E731
    means, quats, scales, opac, tex = (t(scene[k]) for k in ("means", "quats", "scales", "opacity", "texels"))
    spec = torch.cat([t(m).reshape(-1) for m in env["spec"]])
    irr, lut = t(env["irr"]), t(env["lut"])
    sc = P.Scene.from_arrays(scene, env)
    stream = torch.cuda.current_stream()

    for cam in cams:
        ref, _ = P.render(sc, cam)
        out = torch.full((cam["H"], cam["W"], 4), float("nan"), dtype=torch.float32, device=dev)
        c = P.make_camera(cam)
        st = L.ts_render_noalloc(means.shape[0], means.data_ptr(), quats.data_ptr(), scales.data_ptr(),
                                 opac.data_ptr(), tex.shape[1], tex.data_ptr(), len(env["spec"]),
                                 env["spec"][0].shape[1], spec.data_ptr(), irr.shape[1], irr.data_ptr(),
                                 lut.shape[0], lut.data_ptr(), C.byref(c), out.data_ptr(),
                                 C.c_void_p(stream.cuda_stream))
        assert st == 0, L.ts_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert (out[..., 3] > 0).sum() > 100
        assert (out - ref).abs().max().item() <= IMG_TOL


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
