"""Central finite differences of the GPU forward against the GPU backward on
the 200k-splat 800x800 training view: 64 seeded-random parameters, 8 in each
group the paper optimises end to end (Sec. 3.6): centres, rotations, scales,
opacities, albedo texels, roughness / metallic texels, tangent-normal texels
and environment texels (specular and irradiance cubes).

For probe k of parameter theta the objective is S_k = sum_p dL_p . rgba_p over
a probe set P_k of at most 128 pixels where theta acts (the splat's support
square; for a texel, the pixels whose bilinear corners include it), dL random.
The image is piecewise smooth: a step of +-h can carry a pixel across a
discrete decision (support edge, alpha cut, termination, orientation, a
texel or cube cell boundary, a clamp), where the difference quotient sees a
jump or a kink the derivative does not have.  The oracle therefore evaluates
the probe pixels at theta - h and theta + h in FP64 and drops from P_k every
pixel whose discrete state differs between the two, or that lies within FP32
error of a decision at either end (the pixels' admissible-result and
gradient masks).  The GPU gradient is taken with the same dL_k.  Environment
texels enter the colour linearly and change no decision: their probes use
the whole image.  Parameters are drawn among those the view constrains
(full-image gradient at least 1e-2 of the group's largest); one whose step
carries most of its probe pixels across a decision (fewer than 16 left) is
replaced by the next of its group's seeded order.  The difference quotient
is taken at four steps h (1, 1.3, 1.7, 2.2) and the median kept; the
noise term is the larger of the quotients' spread about it and 3 sqrt(sum_p
(dL_p ulp(rgba_p))^2) / (2h) (the float32 rounding of the two forwards,
which no step removes).  Pass: |fd - g| <= 1e-2 |g| + noise.  Each probe's
GPU gradient is also compared with the FP64 oracle's analytic derivative
of the same S_k (autograd on the probe pixels): |g - g64| <= 1e-2 |g64|.
"""
import numpy as np
import pytest
import torch

import scenegen as sg
from oracle import keys as K
from oracle import render as R
from oracle.shading import A_MIN, NDOTV_MIN, cube_face_coords

pytestmark = pytest.mark.gpu

N_PER_GROUP = 8
MAX_PIX = 128
STEPS = {"means": 1e-4, "quats": 5e-4, "scales": 1e-4, "opacity": 1e-3, "albedo": 2e-3, "rough_metal": 2e-3,
         "normal": 2e-3, "env": 1e-2}
MULTS = (1.0, 1.3, 1.7, 2.2)  # step multiples of each probe
ACTIVE = 1e-2  # a parameter the view constrains: |full-image gradient| >= ACTIVE x its group's largest
CHANNELS = {"albedo": (0, 1, 2), "rough_metal": (3, 4), "normal": (5, 6, 7)}


@pytest.fixture(scope="module")
def P():
    import paper_2506_13348_b300 as P
    return P


def shading_signature(X, A, d, env):
    """Discrete state of the shading of each pixel: cube faces and cells of
    the normal and reflection lookups, BRDF-table cells, mip level and the
    clamps (the places where the shaded colour has a kink)."""
    with torch.no_grad():
        ok = A >= A_MIN
        As = torch.where(ok, A, torch.ones_like(A))
        rough = X[:, 4] / As
        N = X[:, 5:8]
        wo = -d / torch.linalg.vector_norm(d, dim=-1, keepdim=True)
        Nh = N / torch.linalg.vector_norm(N, dim=-1, keepdim=True).clamp_min(1e-300)
        nv = (Nh * wo).sum(-1)
        wr = 2.0 * nv[:, None] * Nh - wo
        cols = [ok.long(), (nv < NDOTV_MIN).long(), (rough < 0).long(), (rough > 1).long()]
        Rl = env["lut"].shape[0]
        ndv, rc = nv.clamp(NDOTV_MIN, 1.0), rough.clamp(0.0, 1.0)
        cols += [torch.floor(ndv * Rl - 0.5).long(), torch.floor(rc * Rl - 0.5).long()]
        for dirv, res in ((wr, [m.shape[1] for m in env["spec"]]), (Nh, [env["irr"].shape[1]])):
            f, s, t, _ = cube_face_coords(dirv)
            cols.append(f)
            for r in res:
                cols += [torch.floor(s * r - 0.5).long(), torch.floor(t * r - 0.5).long()]
        if len(env["spec"]) > 1:
            cols.append(torch.floor(rc * float(len(env["spec"]) - 1)).long())
        return torch.stack(cols, -1) * ok[:, None].long()


def sub_scene(scene, ids):
    """The splats `ids` (sorted) as a scene of their own (the oracle's cost
    then scales with the probe's lists, not with the whole scene)."""
    out = {k: np.asarray(scene[k])[ids] for k in ("means", "quats", "scales", "opacity", "texels")}
    out["T"] = scene["T"]
    return out


def oracle_state(scene, cam, env, px, py, kl, T):
    """Per-pixel discrete signature and FP32-band flags of the oracle at the
    probe pixels (lists truncated to the prefix the pixel can still reach)."""
    tiles_x = kl["view"]["tiles_x"]
    full = [R.tile_candidates(kl, (y // 16) * tiles_x + (x // 16)) for x, y in zip(px, py)]
    ids = np.unique(np.concatenate(full))
    params = R.to_params(sub_scene(scene, ids))
    envp = R.env_params(env)
    cands = [np.searchsorted(ids, c) for c in full]

    def run(limit):
        Lm = max(1, min(limit, max(c.size for c in cands)))
        cm = np.full((len(px), Lm), -1, dtype=np.int64)
        for i, c in enumerate(cands):
            cm[i, :min(c.size, Lm)] = c[:Lm]
        fr = R.fragments(params, cam, px, py, torch.from_numpy(cm), R.DEFAULT_MARGINS)
        reached = torch.tensor([c.size > Lm for c in cands]) & (fr["T"] >= R.T_MIN * 0.5)
        return fr, bool(reached.any())

    fr, short = run(1024)
    if short:
        fr, _ = run(1 << 30)
    bl = fr["blended"]
    coord = lambda w: torch.floor((w + 3.0) / 6.0 * T - 0.5).long()  # noqa: E731
    frag = torch.stack([bl.long(), torch.where(bl, coord(fr["u"]), 0), torch.where(bl, coord(fr["v"]), 0),
                        torch.where(bl, (fr["oG"] > R.ALPHA_MAX).long(), 0),
                        torch.where(bl, fr["flip"].long(), 0)], -1)
    sig = (frag.reshape(len(px), -1), shading_signature(fr["X"].detach(), fr["A"].detach(), fr["ray_d"], envp))
    band = fr["decision_band"] | fr["ambiguous"] | fr["kink"]
    return sig, band


def oracle_probe_grad(scene, cam, env, px, py, kl, dl_px, grp, idx):
    """The FP64 oracle's derivative of S = sum_p dL_p . rgba_p over the probe
    pixels with respect to one splat or texel parameter (autograd of the
    plain definition on the splats of the pixels' lists)."""
    tiles_x = kl["view"]["tiles_x"]
    full = [R.tile_candidates(kl, (y // 16) * tiles_x + (x // 16)) for x, y in zip(px, py)]
    ids = np.unique(np.concatenate(full))
    params = R.to_params(sub_scene(scene, ids), requires_grad=True)
    envp = R.env_params(env)
    Lm = max(c.size for c in full)
    cm = np.full((len(px), Lm), -1, dtype=np.int64)
    for i, c in enumerate(full):
        cm[i, :c.size] = np.searchsorted(ids, c)
    fr = R.fragments(params, cam, px, py, torch.from_numpy(cm))
    col = R.shade(fr["X"], fr["A"], fr["ray_d"], envp)
    (col * torch.from_numpy(np.asarray(dl_px, dtype=np.float64))).sum().backward()
    j = int(np.searchsorted(ids, idx[0]))
    key = "texels" if grp in CHANNELS else grp
    return float(params[key].grad[(j,) + tuple(idx[1:])])


def probe_mask(scene_m, scene_p, cam, env, px, py, kl, T):
    """True where the pixel keeps every discrete state across the step and
    sits near no decision at either end."""
    (fa, sa), ba = oracle_state(scene_m, cam, env, px, py, kl, T)
    (fb, sb), bb = oracle_state(scene_p, cam, env, px, py, kl, T)
    L = min(fa.shape[1], fb.shape[1])
    same = (fa[:, :L] == fb[:, :L]).all(1) & (fa[:, L:] == 0).all(1) & (fb[:, L:] == 0).all(1)
    same &= (sa == sb).all(1)
    return (same & ~ba & ~bb).numpy()


def splat_pixels(scene, cam, kl, j, rng):
    """Pixels of splat j's support square inside its tile rectangle and the
    splat's local coordinates there."""
    x0, x1, y0, y1 = kl["view"]["rect"][j]
    xs = np.arange(x0 * 16, min(cam["W"], (x1 + 1) * 16))
    ys = np.arange(y0 * 16, min(cam["H"], (y1 + 1) * 16))
    gy, gx = np.meshgrid(ys, xs, indexing="ij")
    px, py = gx.ravel(), gy.ravel()
    one = R.to_params(sub_scene(scene, np.array([j])))
    fr = R.fragments(one, cam, px, py, torch.zeros((px.size, 1), dtype=torch.long))
    u, v = fr["u"][:, 0].numpy(), fr["v"][:, 0].numpy()
    ok = fr["valid"][:, 0].numpy()
    return px[ok], py[ok], u[ok], v[ok]


def reordered_pixels(scene, cam, kl, j, vm, vp, axis, px, py):
    """Probe pixels where moving splat j's centre from vm to vp along `axis`
    can change the blend order (the GPU sorts again at each step): another
    splat of the pixel's list whose depth key lies between j's two keys and
    that has a fragment there.  They are dropped from the probe."""
    bits = []
    for val in (vm, vp):
        one = {k: np.asarray(scene[k])[j:j + 1].copy() for k in ("means", "quats", "scales", "opacity")}
        one["means"][0, axis] = val
        bits.append(int(K.splat_view_f32(one, cam)["depth_bits"][0]))
    lo, hi = min(bits), max(bits)
    db = kl["view"]["depth_bits"]
    tiles_x = kl["view"]["tiles_x"]
    drop = np.zeros(px.size, bool)
    for i, (x, y) in enumerate(zip(px, py)):
        ids = R.tile_candidates(kl, (y // 16) * tiles_x + (x // 16))
        near = ids[(ids != j) & (db[ids] >= lo) & (db[ids] <= hi)]
        if near.size:
            fr = R.fragments(R.to_params(sub_scene(scene, np.sort(near))), cam, np.array([x]), np.array([y]),
                             torch.arange(near.size)[None])
            drop[i] = bool(fr["valid"].any())
    return drop


def test_gpu_central_differences_64_random_parameters(P):
    scene = sg.make_scene(1)
    env = sg.make_env(1, cube_res=32, levels=1, irr_res=8, lut_res=128)
    cam = sg.fibonacci_cameras(100, 4.0, 800, 800)[17]
    W, H, T = 800, 800, scene["T"]
    dev = torch.device("cuda", 0)
    kl = K.build_keys(scene, cam)
    rng = np.random.default_rng(64)
    sc = P.Scene.from_arrays(scene, env)
    tex_dev = torch.from_numpy(scene["texels"]).to(dev)

    # the parameters that act on this view: non-zero gradient of a full-image
    # random objective
    dl_full = torch.from_numpy(rng.normal(size=(H, W, 4)).astype(np.float32)).to(dev)
    grads = P.zero_grads(sc)
    _, saved = P.render(sc, cam, save=True)
    P.render_backward(saved, dl_full, grads)
    torch.cuda.synchronize()
    g_full = {k: v.detach().cpu().numpy() for k, v in grads.items() if v is not None}

    def candidates(arr, mask=None):
        """A seeded random order of the entries the view constrains."""
        flat = np.abs(arr).ravel()
        ok = flat >= ACTIVE * flat.max() if mask is None else mask.ravel() & (flat >= ACTIVE * flat[mask.ravel()].max())
        return [np.unravel_index(i, arr.shape) for i in rng.permutation(np.nonzero(ok)[0])]

    texg = g_full["texels"].reshape(scene["texels"].shape)
    pools = {}
    for grp in ("means", "quats", "scales", "opacity"):
        pools[grp] = candidates(g_full[grp].reshape(scene[grp].shape))
    for grp, chans in CHANNELS.items():
        m = np.zeros(texg.shape, bool)
        m[..., list(chans)] = True
        pools[grp] = candidates(texg, m)
    pools["env_spec"] = candidates(g_full["spec"].reshape(env["spec"][0].shape))
    pools["env_irr"] = candidates(g_full["irr"].reshape(env["irr"].shape))
    want = {g: N_PER_GROUP for g in pools}
    want["env_spec"] = want["env_irr"] = N_PER_GROUP // 2

    def render_S(dl_img, imgs):
        out, _ = P.render(sc, cam)
        torch.cuda.synchronize()
        imgs.append(out.clone())
        return float((out.double() * dl_img.double()).sum())

    def set_param(grp, idx, val):
        """Writes one float32 value into the GPU scene (and returns the scene
        arrays for the oracle)."""
        s2 = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
        if grp in ("means", "quats", "scales", "opacity"):
            s2[grp][idx] = val
            sc.upload_gaussians(s2["means"], s2["quats"], s2["scales"], s2["opacity"])
        return s2

    def run_probe(grp, idx):
        h = STEPS["env" if grp.startswith("env") else grp]
        if grp in ("means", "quats", "scales", "opacity"):
            px, py, _, _ = splat_pixels(scene, cam, kl, idx[0], rng)
        elif grp in CHANNELS:
            j, tj, ti, _ = idx
            px, py, u, v = splat_pixels(scene, cam, kl, j, rng)
            i0 = np.floor((u + 3.0) / 6.0 * T - 0.5).astype(int)
            j0 = np.floor((v + 3.0) / 6.0 * T - 0.5).astype(int)
            col = (np.clip(i0, 0, T - 1) == ti) | (np.clip(i0 + 1, 0, T - 1) == ti)
            row = (np.clip(j0, 0, T - 1) == tj) | (np.clip(j0 + 1, 0, T - 1) == tj)
            px, py = px[col & row], py[col & row]
        else:
            px = py = None
        if px is not None:
            if px.size > MAX_PIX:
                sel = rng.choice(px.size, MAX_PIX, replace=False)
                px, py = px[sel], py[sel]
            assert px.size > 0, (grp, idx)
        # perturbed values in float32 (the steps actually taken); the masks
        # cover the largest step
        hmax = h * MULTS[-1]
        if grp in ("means", "quats", "scales", "opacity"):
            v0 = np.float32(scene[grp][idx])
            vm, vp = np.float32(v0 - hmax), np.float32(v0 + hmax)
            sm, sp = set_param(grp, idx, vm), set_param(grp, idx, vp)
            keep = probe_mask(sm, sp, cam, env, px, py, kl, T)
            if grp == "means":
                keep &= ~reordered_pixels(scene, cam, kl, idx[0], vm, vp, idx[1], px, py)
        elif grp in CHANNELS:
            v0 = np.float32(scene["texels"][idx])
            vm, vp = np.float32(v0 - hmax), np.float32(v0 + hmax)
            sm = dict(scene, texels=scene["texels"].copy())
            sp = dict(scene, texels=scene["texels"].copy())
            sm["texels"][idx], sp["texels"][idx] = vm, vp
            keep = probe_mask(sm, sp, cam, env, px, py, kl, T)
        else:
            arr = env["spec"][0] if grp == "env_spec" else env["irr"]
            v0 = np.float32(arr[idx])
        # dL on the kept probe pixels (the whole image for the environment)
        dl = np.zeros((H, W, 4), np.float32)
        if px is not None:
            px, py = px[keep], py[keep]
            if px.size < 16:  # the step moves most of the probe across a decision: draw another
                return None
            dl[py, px] = rng.normal(size=(px.size, 4))
        else:
            dl[:] = rng.normal(size=(H, W, 4))
        dlt = torch.from_numpy(dl).to(dev)

        # GPU gradient with this dL
        for v in grads.values():
            if v is not None:
                v.zero_()
        sc.upload_gaussians(scene["means"], scene["quats"], scene["scales"], scene["opacity"])
        _, saved = P.render(sc, cam, save=True)
        P.render_backward(saved, dlt, grads)
        torch.cuda.synchronize()
        saved.release()
        if grp in ("means", "quats", "scales", "opacity"):
            g = float(grads[grp].cpu().numpy().reshape(scene[grp].shape)[idx])
        elif grp in CHANNELS:
            g = float(grads["texels"].cpu().numpy().reshape(scene["texels"].shape)[idx])
        elif grp == "env_spec":
            g = float(grads["spec"].cpu().numpy().reshape(env["spec"][0].shape)[idx])
        else:
            g = float(grads["irr"].cpu().numpy().reshape(env["irr"].shape)[idx])

        # GPU forward at theta -+ h for several steps: the median quotient is
        # the estimate, their spread measures the FP32 noise of the forward
        fds, spread_imgs = [], None
        for mlt in MULTS:
            vm, vp = np.float32(v0 - h * mlt), np.float32(v0 + h * mlt)
            S, imgs = [], []
            for val in (vm, vp):
                if grp in ("means", "quats", "scales", "opacity"):
                    set_param(grp, idx, val)
                elif grp in CHANNELS:
                    t2 = tex_dev.clone()
                    t2[idx] = float(val)
                    sc.upload_atlas(t2, "f32")
                else:
                    e2 = dict(env, spec=[m.copy() for m in env["spec"]], irr=env["irr"].copy())
                    (e2["spec"][0] if grp == "env_spec" else e2["irr"])[idx] = val
                    sc.upload_envmap(e2, "f32")
                S.append(render_S(dlt, imgs))
            fds.append((S[1] - S[0]) / (float(vp) - float(vm)))
            if spread_imgs is None:
                spread_imgs, step = imgs, float(vp) - float(vm)
        # restore
        sc.upload_gaussians(scene["means"], scene["quats"], scene["scales"], scene["opacity"])
        if grp in CHANNELS:
            sc.upload_atlas(tex_dev, "f32")
        if grp.startswith("env"):
            sc.upload_envmap(env, "f32")
        fd = float(np.median(fds))
        spread = float(max(abs(f - fd) for f in fds))
        # FP32 resolution of the two forwards: each value the parameter acts
        # on is rounded to its float32 grid (an ulp of it, uncorrelated
        # between pixels) -- the probe pixels, or for the environment the
        # pixels the step changed
        imgs = spread_imgs
        on = np.zeros((H, W), bool)
        if px is not None:
            on[py, px] = True
        else:
            on = (imgs[0] != imgs[1]).any(-1).cpu().numpy()
        mag = np.maximum(np.abs(imgs[0].cpu().numpy()), np.abs(imgs[1].cpu().numpy())).astype(np.float64)
        ulp = np.spacing(np.maximum(mag[on], 2.0 ** -4).astype(np.float32)).astype(np.float64)
        noise = max(3.0 * float(np.sqrt(((dl[on].astype(np.float64) * ulp) ** 2).sum())) / step, spread)
        tol = 1e-2 * abs(g) + noise
        g64 = oracle_probe_grad(scene, cam, env, px, py, kl, dl[py, px], grp, idx) if px is not None else float("nan")
        return (grp, tuple(int(i) for i in idx), g, fd, abs(fd - g), tol, noise, g64)

    results = []
    for grp, pool in pools.items():
        got = 0
        for idx in pool:
            r = run_probe(grp, idx)
            if r is not None:
                results.append(r)
                got += 1
            if got == want[grp]:
                break
        assert got == want[grp], (grp, got)
    assert len(results) == 64
    for r in results:
        print("[fd] %-12s %-18s g=% .6e fd=% .6e |d|=%.2e tol=%.2e noise=%.2e rel=%.2e oracle=% .6e rel_oracle=%.2e"
              % (r[:7] + (r[4] / max(abs(r[2]), 1e-30), r[7], abs(r[2] - r[7]) / max(abs(r[7]), 1e-30))))
    bad = [r for r in results if not r[4] <= r[5]]
    assert not bad, bad
    # the GPU gradient against the FP64 oracle's on the same probe pixels
    # and dL (not for the environment probes, which span the whole image)
    bad64 = [r for r in results if np.isfinite(r[7]) and not abs(r[2] - r[7]) <= 1e-2 * abs(r[7]) + 1e-6]
    assert not bad64, bad64
    rel = [r[4] / max(abs(r[2]), 1e-30) for r in results if abs(r[2]) > 0]
    print(f"[fd] 64 probes, max rel err {max(rel):.2e}, median {np.median(rel):.2e}")
