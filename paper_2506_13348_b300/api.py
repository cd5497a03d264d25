"""Python binding of the renderer: argument marshalling around the C ABI.

Torch provides device memory and streams; every step of rendering and its
backward runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C
from typing import Sequence

import numpy as np
import torch

from ._lib import TS_BF16, TS_F16, TS_F32, TsCamera, TsFragStats, TsGrads, check, lib

DTYPES = {"f32": TS_F32, "bf16": TS_BF16, "f16": TS_F16, torch.float32: TS_F32, torch.bfloat16: TS_BF16,
          torch.float16: TS_F16}


def _ptr(t) -> C.c_void_p:
    if t is None:
        return C.c_void_p(0)
    return C.c_void_p(t.data_ptr())


def _stream(stream=None) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def make_camera(cam: dict) -> TsCamera:
    c = TsCamera()
    R = np.asarray(cam["R"], dtype=np.float32).reshape(9)
    t = np.asarray(cam["t"], dtype=np.float32).reshape(3)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(t[i])
    c.fx, c.fy, c.cx, c.cy = (float(np.float32(cam[k])) for k in ("fx", "fy", "cx", "cy"))
    c.width, c.height = int(cam["W"]), int(cam["H"])
    vis = cam.get("vis")  # optional [H, W] float32 CUDA tensor: visibility V (Eq. 12)
    if vis is not None:
        assert vis.is_cuda and vis.dtype == torch.float32 and vis.is_contiguous() and tuple(vis.shape) == (c.height, c.width)
        c.visibility = vis.data_ptr()
    return c


def _dev_f32(a, device) -> torch.Tensor:
    if isinstance(a, torch.Tensor):
        return a.detach().to(device=device, dtype=torch.float32).contiguous()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(device)


class Scene:
    """Library-owned splats, texel atlas and environment light on one GPU."""

    def __init__(self, device: int = 0):
        self.device = device
        h = C.c_void_p()
        check(lib().ts_create_scene(C.byref(h), device), "ts_create_scene")
        self.handle = h
        self.n = 0
        self.T = 0
        self.levels = 0
        self.spec_sizes = []
        self.irr_size = 0
        self.normal_encoding = "xyz"

    def close(self):
        if self.handle:
            lib().ts_destroy_scene(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def upload_gaussians(self, means, quats, scales, opacity, stream=None):
        dev = torch.device("cuda", self.device)
        m, q, s, o = (_dev_f32(a, dev) for a in (means, quats, scales, opacity))
        n = m.shape[0]
        check(lib().ts_upload_gaussians(self.handle, n, _ptr(m), _ptr(q), _ptr(s), _ptr(o), 1, _stream(stream)),
              "ts_upload_gaussians")
        self.n = n

    def upload_atlas(self, texels, store="f32", stream=None):
        dev = torch.device("cuda", self.device)
        t = _dev_f32(texels, dev)
        T = t.shape[1]
        check(lib().ts_upload_atlas(self.handle, T, 8, DTYPES[store], _ptr(t), 1, _stream(stream)),
              "ts_upload_atlas")
        self.T = T

    def upload_indirect(self, coeffs, stream=None):
        """Per-splat SH coefficients of the indirect light, [n, K, 3] with K in
        {1, 4, 9} (degree 0-2); None removes them."""
        if coeffs is None:
            check(lib().ts_upload_indirect(self.handle, -1, None, 1, _stream(stream)), "ts_upload_indirect")
            self.sh_K = 0
            return
        t = _dev_f32(coeffs, torch.device("cuda", self.device))
        K = t.shape[1]
        deg = {1: 0, 4: 1, 9: 2}[K]
        check(lib().ts_upload_indirect(self.handle, deg, _ptr(t), 1, _stream(stream)), "ts_upload_indirect")
        self.sh_K = K

    def build_atlas2d(self, store="f32", packing="splat_id", stream=None):
        """Packs the charts into the 2-D hardware-texture atlases (supplementary
        Sec. 1), in splat id order or the Morton order of the splat centres."""
        from ._lib import PACKINGS
        check(lib().ts_scene_build_atlas2d(self.handle, DTYPES[store], PACKINGS[packing], _stream(stream)),
              "ts_scene_build_atlas2d")

    def set_sampler(self, sampler: str):
        """'software' (default), 'hw_atlas' (tex2D on the 2-D atlases) or 'flat'
        (one attribute vector per splat, the untextured baseline)."""
        from ._lib import SAMPLERS
        check(lib().ts_scene_set_sampler(self.handle, SAMPLERS[sampler]), "ts_scene_set_sampler")

    def set_normal_encoding(self, encoding: str):
        """'xyz' (default: three stored tangent-normal components) or 'xy'
        (channels 5-6 hold n_x, n_y; n_z is rebuilt from the interpolated
        pair, Sec. 3.5.1)."""
        from ._lib import NORMAL_ENCODINGS
        check(lib().ts_scene_set_normal_encoding(self.handle, NORMAL_ENCODINGS[encoding]),
              "ts_scene_set_normal_encoding")
        self.normal_encoding = encoding

    def upload_envmap(self, env: dict, store="f32", stream=None):
        dev = torch.device("cuda", self.device)
        spec = [_dev_f32(m, dev) for m in env["spec"]]
        flat = torch.cat([x.reshape(-1) for x in spec])
        irr = _dev_f32(env["irr"], dev)
        lut = _dev_f32(env["lut"], dev)
        check(lib().ts_upload_envmap(self.handle, len(spec), spec[0].shape[1], _ptr(flat), irr.shape[1], _ptr(irr),
                                     lut.shape[0], _ptr(lut), DTYPES[store], 1, _stream(stream)),
              "ts_upload_envmap")
        self.levels = len(spec)
        self.spec_sizes = [x.numel() for x in spec]
        self.irr_size = irr.numel()

    @classmethod
    def from_arrays(cls, scene: dict, env: dict, device: int = 0, store="f32", env_store="f32"):
        s = cls(device)
        s.upload_gaussians(scene["means"], scene["quats"], scene["scales"], scene["opacity"])
        s.upload_atlas(scene["texels"], store)
        s.upload_envmap(env, env_store)
        if "sh" in scene:
            s.upload_indirect(scene["sh"])
        if scene.get("normal_encoding", "xyz") != "xyz":
            s.set_normal_encoding(scene["normal_encoding"])
        return s


class Saved:
    """Forward state kept for the backward (library-owned)."""

    def __init__(self, handle, views):
        self.handle = handle
        self.views = views  # list of (W, H)

    def release(self):
        if self.handle:
            lib().ts_release_saved(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass

    def sizes(self):
        k, t = C.c_int64(), C.c_int64()
        check(lib().ts_saved_sizes(self.handle, C.byref(k), C.byref(t)), "ts_saved_sizes")
        return k.value, t.value

    def lists(self, n_items: int, stream=None):
        K, ntiles = self.sizes()
        ids = torch.empty(max(K, 1), dtype=torch.int32, device="cuda")
        rng = torch.empty(ntiles, 2, dtype=torch.int32, device="cuda")
        db = torch.empty(max(n_items, 1), dtype=torch.int32, device="cuda")
        check(lib().ts_saved_copy_lists(self.handle, _ptr(ids), _ptr(rng), _ptr(db), _stream(stream)),
              "ts_saved_copy_lists")
        torch.cuda.synchronize()
        u32 = lambda t: t.cpu().numpy().view(np.uint32)  # noqa: E731
        return u32(ids)[:K], u32(rng).astype(np.int64), u32(db)[:n_items]

    def pixels(self, view: int = 0, stream=None):
        W, H = self.views[view]
        g = torch.empty(H, W, 8, dtype=torch.float32, device="cuda")
        tr = torch.empty(H, W, dtype=torch.float32, device="cuda")
        last = torch.empty(H, W, dtype=torch.int32, device="cuda")
        check(lib().ts_saved_copy_pixels(self.handle, view, _ptr(g), _ptr(tr), _ptr(last), _stream(stream)),
              "ts_saved_copy_pixels")
        return g, tr, last

    def depth(self, view: int = 0, stream=None):
        """(blended camera depth zsum [H, W], coverage [H, W]) of a view."""
        W, H = self.views[view]
        z = torch.empty(H, W, dtype=torch.float32, device="cuda")
        a = torch.empty(H, W, dtype=torch.float32, device="cuda")
        check(lib().ts_saved_copy_depth(self.handle, view, _ptr(z), _ptr(a), _stream(stream)), "ts_saved_copy_depth")
        return z, a

    def normal_loss(self, loss: torch.Tensor, weight: float = 1.0, view: int = 0, stream=None):
        """weight x L_n (Sec. 3.6) of a view into the device scalar ``loss``;
        its gradient joins the next render_backward of this saved state."""
        check(lib().ts_normal_loss(self.handle, view, float(weight), _ptr(loss), _stream(stream)), "ts_normal_loss")

    def frag_stats(self, stream=None) -> dict:
        st = TsFragStats()
        check(lib().ts_saved_frag_stats(self.handle, C.byref(st), _stream(stream)), "ts_saved_frag_stats")
        return dict(n_pairs=st.n_pairs, n_evaluated=st.n_evaluated, n_blended=st.n_blended,
                    n_visible=st.n_visible, n_texels_read=st.n_texels_read, n_items_blended=st.n_items_blended)


def render(scene: Scene, cam: dict, out: torch.Tensor | None = None, save: bool = False, stream=None):
    """Render one view into ``out`` ([H,W,4] float32 CUDA).  Returns (out, Saved|None)."""
    W, H = int(cam["W"]), int(cam["H"])
    if out is None:
        out = torch.empty(H, W, 4, dtype=torch.float32, device=torch.device("cuda", scene.device))
    c = make_camera(cam)
    h = C.c_void_p()
    check(lib().ts_render(scene.handle, C.byref(c), _ptr(out), C.byref(h) if save else None, _stream(stream)),
          "ts_render")
    return out, (Saved(h, [(W, H)]) if save else None)


def render_views(scenes: Sequence[Scene], cams: Sequence[dict], outs=None, save: bool = False, stream=None):
    """Render a batch of views (one launch sequence).  Returns (outs, Saved|None)."""
    n = len(cams)
    if outs is None:
        outs = [torch.empty(int(c["H"]), int(c["W"]), 4, dtype=torch.float32,
                            device=torch.device("cuda", scenes[i].device)) for i, c in enumerate(cams)]
    carr = (TsCamera * n)(*[make_camera(c) for c in cams])
    sarr = (C.c_void_p * n)(*[s.handle for s in scenes])
    oarr = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    h = C.c_void_p()
    check(lib().ts_render_views(sarr, carr, n, oarr, C.byref(h) if save else None, _stream(stream)),
          "ts_render_views")
    return outs, (Saved(h, [(int(c["W"]), int(c["H"])) for c in cams]) if save else None)


def zero_grads(scene: Scene, device=None) -> dict:
    dev = device or torch.device("cuda", scene.device)
    z = lambda *s: torch.zeros(*s, dtype=torch.float32, device=dev)  # noqa: E731
    out = dict(means=z(scene.n, 3), quats=z(scene.n, 4), scales=z(scene.n, 2), opacity=z(scene.n),
               texels=z(scene.n, scene.T, scene.T, 8), spec=z(sum(scene.spec_sizes)), irr=z(scene.irr_size))
    if getattr(scene, "sh_K", 0):
        out["sh"] = z(scene.n, scene.sh_K, 3)
    return out


def render_backward(saved: Saved, dL_drgba, grads: dict, stream=None):
    """Accumulate gradients of the saved forward into ``grads`` (dict of
    CUDA float32 tensors as from :func:`zero_grads`)."""
    dls = dL_drgba if isinstance(dL_drgba, (list, tuple)) else [dL_drgba]
    dls = [d.contiguous() for d in dls]
    arr = (C.c_void_p * len(dls))(*[d.data_ptr() for d in dls])
    g = TsGrads(*[grads.get(k).data_ptr() if grads.get(k) is not None else None
                  for k in ("means", "quats", "scales", "opacity", "texels", "spec", "irr", "sh")])
    check(lib().ts_render_backward(saved.handle, arr, C.byref(g), _stream(stream)), "ts_render_backward")


def l1_loss(rgba: torch.Tensor, target: torch.Tensor, loss: torch.Tensor, grad: torch.Tensor, stream=None):
    n = rgba.shape[0] * rgba.shape[1]
    check(lib().ts_l1_loss(_ptr(rgba), _ptr(target), n, _ptr(loss), _ptr(grad), _stream(stream)), "ts_l1_loss")


def image_loss(rgba: torch.Tensor, target: torch.Tensor, loss: torch.Tensor, grad: torch.Tensor,
               lambda_dssim: float = 0.2, stream=None):
    """(1 - lambda) L1 + lambda (1 - SSIM) of [H, W, 4] CUDA images into the
    device scalar ``loss``; dL/drgba into ``grad`` (Sec. 3.6)."""
    H, W = rgba.shape[0], rgba.shape[1]
    check(lib().ts_image_loss(_ptr(rgba), _ptr(target), W, H, float(lambda_dssim), _ptr(loss), _ptr(grad),
                              _stream(stream)), "ts_image_loss")


def split_spec(scene: Scene, flat: torch.Tensor):
    """Split a concatenated specular-mip gradient into per-level tensors."""
    out, o = [], 0
    for sz in scene.spec_sizes:
        out.append(flat[o:o + sz])
        o += sz
    return out


def activate(log_scales: torch.Tensor, logit_opacity: torch.Tensor, stream=None):
    """(scales, opacity) = (exp(log_scales), sigmoid(logit_opacity)) by the
    library kernel (ts_activate); CUDA float32 in and out."""
    ls, lo = log_scales.contiguous(), logit_opacity.contiguous()
    s, o = torch.empty_like(ls), torch.empty_like(lo)
    check(lib().ts_activate(lo.numel(), _ptr(ls), _ptr(lo), _ptr(s), _ptr(o), _stream(stream)), "ts_activate")
    return s, o


def activate_backward(scales, opacity, g_scales, g_opacity, stream=None):
    """Chain rule of :func:`activate` (ts_activate_backward)."""
    gls, glo = torch.empty_like(scales), torch.empty_like(opacity)
    check(lib().ts_activate_backward(opacity.numel(), _ptr(scales), _ptr(opacity), _ptr(g_scales.contiguous()),
                                     _ptr(g_opacity.contiguous()), _ptr(gls), _ptr(glo), 0, _stream(stream)),
          "ts_activate_backward")
    return gls, glo


class TexSplatRender(torch.autograd.Function):
    """Differentiable render of one view from the raw optimisation variables
    held by the caller as torch tensors: means, quats (any norm), log_scales,
    logit_opacity, texels, spec (flat, all levels), irr.  The activations run
    in the library (ts_activate), the parameters are copied into ``scene``
    on each forward (device to device) and the backward is the library's
    hand-written adjoint followed by the activations' chain rule.  Because
    each forward re-uploads the scene, a second forward on the same scene
    before the first one's backward invalidates the first (its backward then
    raises TS_ERR_STATE): use one scene per pending forward."""

    @staticmethod
    def forward(ctx, scene: Scene, cam: dict, env_lut, means, quats, log_scales, logit_opacity, texels, spec_flat,
                irr):
        scales, opacity = activate(log_scales, logit_opacity)
        scene.upload_gaussians(means, quats, scales, opacity)
        scene.upload_atlas(texels, "f32")
        levels = scene.levels or 1
        base = int(round((spec_flat.numel() / 18 / sum(4.0 ** -l for l in range(levels))) ** 0.5))
        res = [max(1, base >> l) for l in range(levels)]
        spec, o = [], 0
        for r in res:
            n = 6 * r * r * 3
            spec.append(spec_flat[o:o + n].reshape(6, r, r, 3))
            o += n
        scene.upload_envmap(dict(spec=spec, irr=irr, lut=env_lut))
        out, saved = render(scene, cam, save=True)
        ctx.scene = scene
        ctx.saved = saved
        ctx.irr_shape = irr.shape
        ctx.save_for_backward(scales, opacity)
        return out

    @staticmethod
    def backward(ctx, g):
        scene = ctx.scene
        scales, opacity = ctx.saved_tensors
        grads = zero_grads(scene)
        render_backward(ctx.saved, g.contiguous(), grads)
        ctx.saved.release()
        g_ls, g_lo = activate_backward(scales, opacity, grads["scales"], grads["opacity"])
        return (None, None, None, grads["means"], grads["quats"], g_ls, g_lo, grads["texels"], grads["spec"],
                grads["irr"].reshape(ctx.irr_shape))


class Server:
    """Continuous-batching view server (library worker threads and streams).

    ``submit`` returns a ticket at once; ``wait`` returns the image.  Scenes
    must stay alive while their requests are pending."""

    def __init__(self, device: int = 0, arena_bytes: int = 8 << 30, n_streams: int = 2, max_batch: int = 8):
        from ._lib import TsServeStats  # noqa: F401
        h = C.c_void_p()
        check(lib().ts_server_create(C.byref(h), device, arena_bytes, n_streams, max_batch), "ts_server_create")
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            lib().ts_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, scene: Scene, cam: dict) -> int:
        c = make_camera(cam)
        t = C.c_uint64()
        check(lib().ts_server_submit(self.handle, scene.handle, C.byref(c), C.byref(t)), "ts_server_submit")
        return t.value

    def wait(self, ticket: int, out: torch.Tensor | None = None, timeout_s: float = 60.0):
        """Copies the result into ``out`` (CUDA or CPU float32 [H,W,4]);
        returns ``out``.  ``out=None`` discards the image."""
        ptr = C.c_void_p(out.data_ptr()) if out is not None else C.c_void_p(0)
        on_dev = 1 if (out is not None and out.is_cuda) else 0
        check(lib().ts_server_wait(self.handle, C.c_uint64(ticket), ptr, on_dev, C.c_double(timeout_s)),
              "ts_server_wait")
        return out

    def stats(self) -> dict:
        from ._lib import TsServeStats
        s = TsServeStats()
        check(lib().ts_server_stats(self.handle, C.byref(s)), "ts_server_stats")
        return {k: getattr(s, k) for k, _ in TsServeStats._fields_}

    def reset_stats(self):
        check(lib().ts_server_reset_stats(self.handle), "ts_server_reset_stats")

    def request_bytes(self, scene: Scene, cam: dict) -> int:
        """The bytes a request would be admitted with now."""
        c = make_camera(cam)
        b = C.c_size_t()
        check(lib().ts_server_request_bytes(self.handle, scene.handle, C.byref(c), C.byref(b)),
              "ts_server_request_bytes")
        return b.value

    def batch_log(self, max_entries: int = 4096) -> list:
        """[(worker, views, t0_ms, t1_ms)] of the last batches, oldest first
        (device-time intervals, see ts_server_batch_log)."""
        import numpy as np
        w = np.zeros(max_entries, np.int32)
        v = np.zeros(max_entries, np.int32)
        t0 = np.zeros(max_entries, np.float64)
        t1 = np.zeros(max_entries, np.float64)
        n = C.c_int32()
        check(lib().ts_server_batch_log(self.handle, max_entries, C.byref(n), w.ctypes.data, v.ctypes.data,
                                        t0.ctypes.data, t1.ctypes.data), "ts_server_batch_log")
        return [(int(w[i]), int(v[i]), float(t0[i]), float(t1[i])) for i in range(n.value)]


def adam_update(param: torch.Tensor, grad: torch.Tensor, m: torch.Tensor, v: torch.Tensor, step: int,
                lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-15, shadow_ptr: int = 0,
                shadow_dtype="f32", zero_grad: bool = True, stream=None):
    """One fused Adam step in the library (see ts_adam_update)."""
    from ._lib import TsAdam
    hp = TsAdam(lr, beta1, beta2, eps, step)
    check(lib().ts_adam_update(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(), C.byref(hp),
                               C.c_void_p(shadow_ptr), DTYPES[shadow_dtype], 1 if zero_grad else 0,
                               _stream(stream)), "ts_adam_update")


def scene_texels(scene: Scene):
    """(device pointer, T, dtype code) of the scene's stored atlas."""
    p, T, dt = C.c_void_p(), C.c_int(), C.c_int()
    check(lib().ts_scene_texels(scene.handle, C.byref(p), C.byref(T), C.byref(dt)), "ts_scene_texels")
    return p.value, T.value, dt.value


def scene_envmap(scene: Scene):
    """(spec pointer, irr pointer, dtype code) of the scene's stored environment."""
    sp, ir, dt = C.c_void_p(), C.c_void_p(), C.c_int()
    check(lib().ts_scene_envmap(scene.handle, C.byref(sp), C.byref(ir), C.byref(dt)), "ts_scene_envmap")
    return sp.value, ir.value, dt.value


class Trainer:
    """Multi-view training step on one scene, all in library kernels: a
    batched forward of V views (saved state), the loss of each view (L1, or
    L1 + D-SSIM, plus the normal-consistency term when asked), one
    backward over the batch, then Adam on float32 masters of geometry and
    texels with the texel master written back into the scene's stored atlas
    (bf16 / f16 / f32) and the geometry updated in place.  Optionally the
    environment (every specular level and the irradiance cube, written back
    into the scene's stored cubes) and the per-splat SH of the indirect light
    are optimised too, as in Sec. 3.6."""

    def __init__(self, scene: Scene, data: dict, store: str = "bf16", lr_geom: float = 1e-4,
                 lr_tex: float = 1e-2, lambda_dssim: float = 0.0, normal_weight: float = 0.0,
                 env: dict | None = None, lr_env: float = 0.0, lr_sh: float = 0.0):
        """lambda_dssim > 0 trains on (1 - lambda) L1 + lambda D-SSIM and
        normal_weight > 0 adds normal_weight x L_n (the paper's objective,
        Sec. 3.6: lambda 0.2); the defaults keep the plain L1 loss.
        lr_env > 0 optimises the environment maps, starting from ``env`` (the
        dict the scene's environment was uploaded from); lr_sh > 0 optimises
        data["sh"] (the scene must carry SH of that shape)."""
        dev = torch.device("cuda", scene.device)
        f = lambda a: _dev_f32(a, dev).clone()  # noqa: E731
        self.scene, self.store = scene, store
        self.master = dict(means=f(data["means"]), quats=f(data["quats"]), scales=f(data["scales"]),
                           opacity=f(data["opacity"]), texels=f(data["texels"]))
        self.lr = dict(means=lr_geom, quats=lr_geom, scales=lr_geom, opacity=lr_geom, texels=lr_tex)
        if lr_env > 0.0:
            if env is None:
                raise ValueError("Trainer: lr_env needs the initial environment (env=...)")
            self.master["spec"] = torch.cat([f(m).reshape(-1) for m in env["spec"]])
            self.master["irr"] = f(env["irr"]).reshape(-1)
            self.lr["spec"] = self.lr["irr"] = lr_env
        if lr_sh > 0.0:
            if not getattr(scene, "sh_K", 0) or "sh" not in data:
                raise ValueError("Trainer: lr_sh needs a scene with SH and data['sh']")
            self.master["sh"] = f(data["sh"])
            self.lr["sh"] = lr_sh
        self.m = {k: torch.zeros_like(t) for k, t in self.master.items()}
        self.v = {k: torch.zeros_like(t) for k, t in self.master.items()}
        self.grads = zero_grads(scene)
        for k in ("spec", "irr"):
            if k in self.master and self.master[k].numel() != self.grads[k].numel():
                raise ValueError(f"Trainer: env['{k}'] does not match the scene's environment")
        self.step_count = 0
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.lambda_dssim, self.normal_weight = float(lambda_dssim), float(normal_weight)

    def step(self, cams, targets, outs=None, dls=None):
        """One step over the views ``cams`` with target images ``targets``
        ([H,W,4] CUDA each).  Returns the per-view loss tensor (device)."""
        n = len(cams)
        outs, saved = render_views([self.scene] * n, cams, outs=outs, save=True)
        if dls is None:
            dls = [torch.empty_like(o) for o in outs]
        losses = torch.zeros(n, dtype=torch.float32, device=outs[0].device)
        for i in range(n):
            if self.lambda_dssim > 0.0:
                image_loss(outs[i], targets[i], losses[i:i + 1], dls[i], self.lambda_dssim)
            else:
                l1_loss(outs[i], targets[i], losses[i:i + 1], dls[i])
        if self.normal_weight > 0.0:
            ln = torch.zeros(1, dtype=torch.float32, device=outs[0].device)
            for i in range(n):
                saved.normal_loss(ln, self.normal_weight, view=i)
                losses[i:i + 1] += ln
        render_backward(saved, dls, self.grads)
        saved.release()
        self.step_count += 1
        codes = {0: "f32", 1: "bf16", 2: "f16"}
        tex_ptr, _, dt = scene_texels(self.scene)
        shadow = {"texels": (tex_ptr, codes[dt])}
        if "spec" in self.master:
            sp, ir, edt = scene_envmap(self.scene)
            shadow["spec"], shadow["irr"] = (sp, codes[edt]), (ir, codes[edt])
        for k in self.master:
            ptr, sdt = shadow.get(k, (0, "f32"))
            adam_update(self.master[k], self.grads[k], self.m[k], self.v[k], self.step_count, self.lr[k],
                        shadow_ptr=ptr, shadow_dtype=sdt)
        ms = self.master
        check(lib().ts_scene_set_geometry(self.scene.handle, _ptr(ms["means"]), _ptr(ms["quats"]),
                                          _ptr(ms["scales"]), _ptr(ms["opacity"]), _stream(None)),
              "ts_scene_set_geometry")
        if "sh" in ms:  # same degree and count: an in-place, stream-ordered copy
            check(lib().ts_upload_indirect(self.scene.handle, {1: 0, 4: 1, 9: 2}[self.scene.sh_K], _ptr(ms["sh"]), 1,
                                           _stream(None)), "ts_upload_indirect")
        for k in ("spec", "irr", "sh"):  # not optimised: drop the accumulated gradient
            if k not in ms and k in self.grads:
                self.grads[k].zero_()
        return losses
