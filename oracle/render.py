"""FP64 forward renderer of textured 2D Gaussian splats (TEST INFRASTRUCTURE).

The plain definition, evaluated per pixel and per candidate splat, in float64
torch CPU ops (no tiling tricks beyond taking each pixel's candidates from its
tile's sorted list, which the brute-force mode replaces by every visible
splat):

  ray        o + tau d through the pixel centre (x+0.5, y+0.5),
             d = R^T K^-1 (x, y, 1) so that tau is the camera depth
  splat      P_k(u,v) = p_k + s_u t_u u + s_v t_v v, n_k = t_u x t_v  (Sec. 3.1, Eq. 1)
  hit        tau = (p - o).n / d.n, skip if |d.n| <= 1e-12 |d| or tau <= 0.2
  (u, v)     u = (X - p).t_u / s_u, v = (X - p).t_v / s_v   (exact ray-splat intersection)
  support    fragment only if |u| <= 3 and |v| <= 3 (S_sigma = 3, Sec. 3.3)
  kernel     G = exp(-(u^2+v^2)/2)                         (Eq. 2)
  opacity    alpha = min(0.99, o G); skip if alpha < 1/255
  texture    s = (u+3)/6, t = (v+3)/6                      (Eq. 5)
             a = BilinearFilter(T_k, s, t)                 (Eq. 4, Eq. 6)
             texel centres at (i+0.5)/T, clamp-to-edge inside the splat's texture
  normals    n = R_k n^t with R_k = [t_u, t_v, n_k'] and n_k' the splat normal
             turned to face the camera                    (Eq. 7)
             with the two-component encoding (scene["normal_encoding"] ==
             "xy", Sec. 3.5.1) only channels 5-6 are read and
             n^t = (n_x, n_y, sqrt(max(0, 1 - n_x^2 - n_y^2))) from the
             interpolated (n_x, n_y): the paper gives the formula, not
             whether it applies before or after filtering; a filtered
             two-channel texture gives this order
  blending   X = sum_i x_i alpha_i prod_{j<i}(1 - alpha_j)  (Eq. 3, Eq. 8-9)
             A = sum_i alpha_i prod_{j<i}(1 - alpha_j); stop after the first
             fragment that brings the transmittance below 1e-4
  depth      Z = sum_i w_i tau_i (blended camera depth of the hits)
  indirect   with per-splat SH coefficients c_k (degree <= 2; the paper
             defers the SH to Ref-Gaussian without the degree, basis or where
             it is evaluated): l_i = c_k . Y(w_r,i), w_r,i the reflection of
             w_o = -d/|d| about the fragment's normalised normal;
             Xind = sum_i w_i l_i (Eq. 9)
  shading    see shading.py                               (Eq. 10-12)

Products along a pixel's list are cumulative products and sums cumulative sums
(sequential, in list order), so adding a candidate that does not contribute
changes no bit of the result: that is what makes the brute-force comparison
exact.

Admissible results: the definition's thresholds (|u|, |v| <= 3, alpha >=
1/255, T < 1e-4, the orientation test) are discontinuous, and an FP32
renderer evaluating the same definition may land on the other side of one
when the FP64 value lies within FP32 error of it.  Each pixel is classified:
no decision within its band (a unique result), exactly one (two admissible
results: the definition's, and "alt" with that one decision flipped), or
more than one ("ambiguous", masked in comparisons).  Band half-widths are
DEFAULT_MARGINS below.

Parity: pinned by the closed-form single-splat and two-splat tests, the
texel-centre and affine-texture tests, the constant-texture invariant, the
90-degree twist invariant and the brute-force comparison
(tests/test_oracle_render.py); the alternative results by closed forms of
pixels placed exactly at a support edge and at the termination threshold
(tests/test_oracle_alternates.py).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import keys as K
from .shading import shade, shading_ambiguity, shading_kinks

F64 = torch.float64
ALPHA_MIN = float(K.ALPHA_MIN)
ALPHA_MAX = float(np.float32(0.99))
T_MIN = float(np.float32(1e-4))
NEAR = float(K.NEAR)


def to_params(scene: dict, requires_grad: bool = False) -> dict:
    """Float64 torch leaves of the splat parameters (and of the per-splat
    indirect-light SH coefficients 'sh' [n, K, 3] when the scene has them)."""
    out = {}
    for k in ("means", "quats", "scales", "opacity", "texels") + (("sh",) if "sh" in scene else ()):
        t = torch.from_numpy(np.asarray(scene[k], dtype=np.float64).copy())
        t.requires_grad_(requires_grad)
        out[k] = t
    out["normal_xy"] = scene.get("normal_encoding", "xyz") == "xy"
    return out


def env_params(env: dict, requires_grad: bool = False) -> dict:
    spec = []
    for m in env["spec"]:
        t = torch.from_numpy(np.asarray(m, dtype=np.float64).copy())
        t.requires_grad_(requires_grad)
        spec.append(t)
    irr = torch.from_numpy(np.asarray(env["irr"], dtype=np.float64).copy()).requires_grad_(requires_grad)
    lut = torch.from_numpy(np.asarray(env["lut"], dtype=np.float64).copy())
    return dict(spec=spec, irr=irr, lut=lut)


def rotation_columns(q: torch.Tensor):
    """Unit-quaternion rotation matrix columns (t_u, t_v, n) in float64."""
    qn = q / torch.linalg.vector_norm(q, dim=-1, keepdim=True)
    w, x, y, z = qn.unbind(-1)
    tu = torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)], -1)
    tv = torch.stack([2 * (x * y - w * z), 1 - 2 * (x * x + z * z), 2 * (y * z + w * x)], -1)
    n = torch.stack([2 * (x * z + w * y), 2 * (y * z - w * x), 1 - 2 * (x * x + y * y)], -1)
    return tu, tv, n


def camera_tensors(cam: dict):
    R = torch.tensor(np.asarray(cam["R"], dtype=np.float64))
    t = torch.tensor(np.asarray(cam["t"], dtype=np.float64))
    origin = -(R.T @ t)
    return R, t, origin


def pixel_rays(cam: dict, px: np.ndarray, py: np.ndarray) -> torch.Tensor:
    """World-space ray directions through pixel centres; camera-z component 1."""
    R, _, _ = camera_tensors(cam)
    xc = (torch.tensor(px, dtype=F64) + 0.5 - float(cam["cx"])) / float(cam["fx"])
    yc = (torch.tensor(py, dtype=F64) + 0.5 - float(cam["cy"])) / float(cam["fy"])
    dc = torch.stack([xc, yc, torch.ones_like(xc)], -1)
    return dc @ R  # R^T dc, row-vector form


def fragments(params: dict, cam: dict, px, py, cand: torch.Tensor, margins=None):
    """All per-fragment quantities for pixels (px, py) [P] and candidate splat
    indices cand [P, L] (-1 = padding), in list order.

    Returns a dict with alpha-validity masks, the blended weights, the
    per-fragment attribute vectors and the composited G-buffer.  With
    ``margins`` it also classifies each pixel by the discrete decisions of
    the definition (support edge, alpha threshold, termination, orientation)
    that lie within FP32 error of flipping: with none the result is unique;
    with exactly one, flipping that decision gives the only other admissible
    result, returned as ``alt`` (an FP32 renderer may take either branch);
    with more, the pixel is ``ambiguous`` (excluded from comparisons).
    """
    P, L = cand.shape
    _, _, origin = camera_tensors(cam)
    d = pixel_rays(cam, px, py)  # [P,3]
    pad = cand < 0
    ci = cand.clamp_min(0)
    T = params["texels"].shape[1]
    m_uv = margins[0] if margins is not None else 0.0

    tu_all, tv_all, n_all = rotation_columns(params["quats"])
    p = params["means"][ci]          # [P,L,3]
    tu, tv, n = tu_all[ci], tv_all[ci], n_all[ci]
    su = params["scales"][ci][..., 0]
    sv = params["scales"][ci][..., 1]
    op = params["opacity"][ci]

    dd = d[:, None, :]
    den = (dd * n).sum(-1)                       # d.n
    po = p - origin                              # p - o
    num = (po * n).sum(-1)                       # (p - o).n
    dnorm = torch.linalg.vector_norm(d, dim=-1)[:, None]
    hit = (den.abs() > 1e-12 * dnorm) & ~pad
    den_s = torch.where(hit, den, torch.ones_like(den))
    tau = num / den_s
    hit = hit & (tau > NEAR)
    rel = tau[..., None] * dd - po               # X - p
    u = (rel * tu).sum(-1) / su
    v = (rel * tv).sum(-1) / sv
    inside = hit & (u.abs() <= 3.0) & (v.abs() <= 3.0)
    # fragments are also evaluated just outside the support square (within
    # the edge band) so that the alternative with the edge decision flipped
    # can be composited; they carry no weight in the definition's result
    reach = hit & (u.abs() <= 3.0 + m_uv) & (v.abs() <= 3.0 + m_uv)
    u_s = torch.where(reach, u, torch.zeros_like(u))
    v_s = torch.where(reach, v, torch.zeros_like(v))
    G = torch.exp(-(u_s * u_s + v_s * v_s) / 2.0)
    oG = op * G
    alpha = torch.clamp(oG, max=ALPHA_MAX)
    valid = inside & (alpha >= ALPHA_MIN)

    # texture lookup (Eq. 5-6)
    s = (u_s + 3.0) / 6.0
    t = (v_s + 3.0) / 6.0
    from .shading import bilinear_2d
    tex = bilinear_2d(params["texels"], s * T - 0.5, t * T - 0.5, lead_index=ci)  # [P,L,8]

    nt = tex[..., 5:8]
    nz_r = None
    if params.get("normal_xy", False):
        # two stored components (Sec. 3.5.1): n_z from the interpolated
        # (n_x, n_y); zero (and a zero derivative) outside the unit disc
        nz_r = 1.0 - tex[..., 5] * tex[..., 5] - tex[..., 6] * tex[..., 6]
        pos = nz_r > 0.0
        nz = torch.where(pos, torch.sqrt(torch.where(pos, nz_r, torch.ones_like(nz_r))), torch.zeros_like(nz_r))
        nt = torch.cat([tex[..., 5:7], nz[..., None]], -1)
    wo = None
    if "sh" in params:
        from .shading import sh_basis
        wo = -(d / torch.linalg.vector_norm(d, dim=-1, keepdim=True))[:, None, :]
        sh = params["sh"][ci]                                   # [P,L,K,3]

    def composite(valid_, flip_, tmin):
        """Normal mapping and front-to-back compositing of the fragments
        marked valid, with the splat normals flipped where flip_ and the
        termination threshold tmin (a float or a [P, 1] tensor)."""
        # normal mapping (Eq. 7): columns t_u, t_v and the camera-facing normal
        n_face = torch.where(flip_[..., None], -n, n)
        n_w = nt[..., 0:1] * tu + nt[..., 1:2] * tv + nt[..., 2:3] * n_face
        x = torch.cat([tex[..., 0:5], n_w], -1)  # [P,L,8]
        # compositing (Eq. 3, Eq. 8): sequential products / sums along the list
        a = torch.where(valid_, alpha, torch.zeros_like(alpha))
        trans = torch.cumprod(1.0 - a, dim=1)
        T_before = torch.cat([torch.ones_like(trans[:, :1]), trans[:, :-1]], 1)
        blended = valid_ & (T_before >= tmin)
        w = torch.where(blended, a * T_before, torch.zeros_like(a))
        X = torch.cumsum(w[..., None] * x, dim=1)[:, -1, :] if L > 0 else torch.zeros(P, 8, dtype=F64)
        A = torch.cumsum(w, dim=1)[:, -1] if L > 0 else torch.zeros(P, dtype=F64)
        # depth channel: the blended camera depth of the hits, sum_i w_i tau_i
        # (the ray has camera-space z component 1, so tau is the camera depth)
        tau_s = torch.where(blended, tau, torch.zeros_like(tau))
        Z = torch.cumsum(w * tau_s, dim=1)[:, -1] if L > 0 else torch.zeros(P, dtype=F64)
        Xind = None
        if "sh" in params:
            # indirect light (Sec. 3.5, Eq. 9 and 12): each fragment evaluates
            # its splat's SH coefficients in the reflection direction of its
            # own (normal-mapped, normalised) normal; the results are blended
            nl = torch.linalg.vector_norm(n_w, dim=-1, keepdim=True)
            nzm = nl >= 1e-12
            nh = torch.where(nzm, n_w / torch.where(nzm, nl, torch.ones_like(nl)), wo.expand_as(n_w))
            ndw = (nh * wo).sum(-1, keepdim=True)
            wr = 2.0 * ndw * nh - wo
            Y = sh_basis(wr, sh.shape[-2])                          # [P,L,K]
            li = (Y[..., None] * sh).sum(-2)                        # [P,L,3]
            Xind = torch.cumsum(w[..., None] * li, dim=1)[:, -1, :] if L > 0 else torch.zeros(P, 3, dtype=F64)
        ab = torch.where(blended, a, torch.zeros_like(a))
        T_final = torch.cumprod(1.0 - ab, dim=1)[:, -1] if L > 0 else torch.ones(P, dtype=F64)
        idx = torch.arange(L).expand(P, L)
        last = torch.where(blended, idx, torch.full_like(idx, -1)).max(1).values if L > 0 \
            else torch.full((P,), -1, dtype=torch.long)
        return dict(X=X, A=A, Z=Z, Xind=Xind, T=T_final, blended=blended, T_before=T_before, a=a, last=last)

    flip = num > 0.0
    base = composite(valid, flip, T_MIN)
    blended, T_before = base["blended"], base["T_before"]
    out = dict(X=base["X"], A=base["A"], Z=base["Z"], Xind=base["Xind"], T=base["T"], ray_d=d, blended=blended,
               valid=valid, T_before=T_before)
    with torch.no_grad():
        evaluated = (T_before >= T_MIN) & ~pad
        out["n_eval"] = evaluated.sum(1)
        out["n_contrib"] = blended.sum(1)
        # index (within the list) of the last blended fragment, -1 if none
        out["last"] = base["last"]
        # per-fragment local coordinates, unclamped opacity and orientation
        # (for tests that compare discrete states of two evaluations)
        out["u"], out["v"], out["oG"], out["flip"] = u.detach(), v.detach(), oG.detach(), flip
        if margins is not None:
            m_uv, m_a, m_t, m_f = margins
            oG_full = op * torch.exp(-(u * u + v * v).clamp(max=1e4) / 2.0)
            near_edge = (((u.abs() - 3.0).abs() <= m_uv) & (v.abs() <= 3.0 + m_uv)) | \
                        (((v.abs() - 3.0).abs() <= m_uv) & (u.abs() <= 3.0 + m_uv))

            def bands(valid_, res):
                """Fragments whose existence (support edge, alpha threshold),
                termination test or orientation lies within its band, among
                those an FP32 renderer could still evaluate."""
                maybe_eval = (res["T_before"] >= T_MIN * (1.0 - m_t)) & hit
                b_valid = near_edge & (oG_full >= ALPHA_MIN * (1.0 - m_a))
                b_valid |= inside & ((oG - ALPHA_MIN).abs() <= m_a * ALPHA_MIN)
                T_after = res["T_before"] * (1.0 - res["a"])
                b_term = valid_ & ((T_after / T_MIN - 1.0).abs() <= m_t)
                b_flip = inside & (num.abs() <= m_f * torch.linalg.vector_norm(po, dim=-1))
                return b_valid & maybe_eval, b_term & maybe_eval, b_flip & maybe_eval, T_after

            b_valid, b_term, b_flip, T_after = bands(valid, base)
            any_b = b_valid | b_term | b_flip
            n_amb = any_b.sum(1)
            single = n_amb == 1
            # the one alternative: flip that decision (validity, the normal's
            # orientation, or whether compositing stops after the fragment)
            tog_v = b_valid & single[:, None]
            tog_f = b_flip & single[:, None]
            term = b_term & single[:, None] & ~tog_v & ~tog_f
            Ta = torch.where(term, T_after, torch.zeros_like(T_after)).sum(1, keepdim=True)
            has_t = term.any(1, keepdim=True)
            stops = Ta < T_MIN  # the definition stops after it: the alternative goes on for one more
            tmin_alt = torch.where(has_t, torch.where(stops, Ta, Ta * (1.0 + 1e-12)),
                                   torch.full_like(Ta, T_MIN))
            alt = composite(valid ^ tog_v, flip ^ tog_f, tmin_alt)
            # the alternative must not itself sit near another decision
            a_valid, a_term, a_flip, _ = bands(valid ^ tog_v, alt)
            extra = ((a_valid | a_term | a_flip) & ~(tog_v | tog_f | term)).any(1)
            out["alt"] = {k: alt[k] for k in ("X", "A", "Z", "Xind", "T", "last")}
            out["alt_mask"] = single & ~extra
            out["ambiguous"] = (n_amb >= 2) | (single & extra)
            out["decision_band"] = n_amb >= 1
            # derivative kinks of blended fragments (value continuous, slope
            # not): bilinear cell boundaries at texel centres (incl. the
            # clamp edges) and the 0.99 opacity clamp
            m_k = KINK_TEX * max(1.0, T / 8.0)  # texel coordinate = (u + 3) T / 6 - 1/2: error grows with T
            kink = torch.zeros_like(blended)
            for coord in (s * T - 0.5, t * T - 0.5):
                fr_ = coord - torch.floor(coord)
                near = (fr_ <= m_k) | (fr_ >= 1.0 - m_k)
                kink |= near & (coord >= -m_k) & (coord <= T - 1 + m_k)
            kink |= (oG - ALPHA_MAX).abs() <= m_a * ALPHA_MAX
            # nearly edge-on splats (|n . d| <= EDGE_ON_COS |d|):
            # d(u,v)/d(params) grows like 1/cos^2 and an FP32 evaluation
            # keeps only a few correct digits of those gradients
            kink |= den.abs() <= EDGE_ON_COS * dnorm
            if nz_r is not None:  # the n_z reconstruction's clamp at the unit circle
                kink |= nz_r.abs() <= 1e-6
            out["kink"] = (kink & blended).any(1)
    return out


# Half-widths (in texel units) of the bands around texture-lookup kinks that
# the gradient comparison excludes: FP32 (u, v) error ~1e-6 relative maps to
# ~4e-6 texel at T = 8; the band is KINK_TEX at T <= 8 and grows as T / 8
# beyond (the texel coordinate scales u by T / 6).
KINK_TEX = 1e-5
# |cos| between view ray and splat normal below which gradients are excluded
# (~1.15 deg from edge-on).  The local coordinates (u, v) of a hit carry an
# FP32 error that grows like 1/|cos| whichever way they are evaluated (an
# FP32 homography and an FP32 ray-plane evaluation of the same fragments
# measure the same error in every |cos| band: median 4e-5 at |cos| in
# [0.01, 0.03) against 2e-6 above 0.3), and their derivatives grow like
# 1/cos^2, so geometry gradients of fragments this close to edge-on keep only
# a few correct digits.  The band is the narrowest of {0, 0.005, 0.01, 0.02,
# 0.03} at which the 200k-splat scene's 1k-splat slice keeps every gradient
# group within 1e-3 of its maximum (quaternions 6.5e-4 at 0.02, 1.7e-3 at 0.01).
EDGE_ON_COS = 0.02


def tile_candidates(keylist: dict, tile: int) -> np.ndarray:
    s, e = keylist["tile_ranges"][tile]
    return keylist["ids"][s:e].astype(np.int64)


def brute_candidates(view: dict) -> np.ndarray:
    """Every visible splat, ordered by (depth bits, id): the tile-free list."""
    vis = np.nonzero(view["visible"])[0]
    order = np.lexsort((vis, view["depth_bits"][vis]))
    return vis[order].astype(np.int64)


# Margins of the ambiguity mask, chosen from FP32 error bounds of a renderer
# that evaluates the same definition in single precision: (u, v) carry ~1e-6
# relative error (band 3e-5 in u around the support edge), alpha ~1e-6
# relative (band 1e-5), the transmittance after tens of blends ~1e-5
# relative (band 2e-4 around the 1e-4 threshold), and the orientation test
# d.n changes sign only for splats seen within 1e-7 of edge-on.
DEFAULT_MARGINS = (3e-5, 1e-5, 2e-4, 1e-7)


def render(scene: dict, cam: dict, env: dict, *, params=None, envp=None, brute=False,
           tiles=None, margins=DEFAULT_MARGINS, max_entries=4_000_000, keylist=None, vis=None) -> dict:
    """Render the view (or the listed ``tiles``) in float64.

    With per-splat SH in the scene ('sh' [n, K, 3]) the fragments also blend
    their indirect light (Xind [H,W,3]) and ``vis`` [H,W] (visibility V,
    default 1) mixes it into the specular term.
    Returns rgba [H,W,4], the G-buffer X [H,W,8], A, the blended depth Z
    (sum of alpha T times the hit's camera depth), T_final, the ambiguity
    mask, fragment counts (evaluated / contributing), the last contributor
    index and the key list.  With ``params``/``envp`` (torch leaves) the
    images are differentiable.
    """
    W, H = int(cam["W"]), int(cam["H"])
    if params is None:
        params = to_params(scene)
    if envp is None:
        envp = env_params(env)
    kl = keylist if keylist is not None else K.build_keys(scene, cam)
    tiles_x, tiles_y = kl["view"]["tiles_x"], kl["view"]["tiles_y"]
    tile_list = list(range(tiles_x * tiles_y)) if tiles is None else list(tiles)
    brute_list = brute_candidates(kl["view"]) if brute else None

    rgba = torch.zeros(H, W, 4, dtype=F64)
    Xb = torch.zeros(H, W, 8, dtype=F64)
    Ab = torch.zeros(H, W, dtype=F64)
    Zb = torch.zeros(H, W, dtype=F64)
    Ib = torch.zeros(H, W, 3, dtype=F64)
    vis_t = None if vis is None else torch.from_numpy(np.asarray(vis, dtype=np.float64))
    Tb = torch.ones(H, W, dtype=F64)
    amb = torch.zeros(H, W, dtype=torch.bool)
    gamb = torch.zeros(H, W, dtype=torch.bool)
    n_eval = torch.zeros(H, W, dtype=torch.long)
    n_con = torch.zeros(H, W, dtype=torch.long)
    last = torch.full((H, W), -1, dtype=torch.long)
    covered = torch.zeros(H, W, dtype=torch.bool)
    alt = dict(rgba=torch.zeros(H, W, 4, dtype=F64), X=torch.zeros(H, W, 8, dtype=F64),
               A=torch.zeros(H, W, dtype=F64), Z=torch.zeros(H, W, dtype=F64), T=torch.ones(H, W, dtype=F64),
               last=torch.full((H, W), -1, dtype=torch.long), mask=torch.zeros(H, W, dtype=torch.bool))

    def run_chunk(chunk):
        pxs, pys, cands = [], [], []
        for tl in chunk:
            tx, ty = tl % tiles_x, tl // tiles_x
            xs = np.arange(tx * K.TILE, min(W, (tx + 1) * K.TILE))
            ys = np.arange(ty * K.TILE, min(H, (ty + 1) * K.TILE))
            gy, gx = np.meshgrid(ys, xs, indexing="ij")
            c = brute_list if brute else tile_candidates(kl, tl)
            pxs.append(gx.ravel())
            pys.append(gy.ravel())
            cands.append(np.broadcast_to(c, (gx.size, c.size)))
        Lm = max(c.shape[1] for c in cands)
        Pn = sum(c.shape[0] for c in cands)
        cm = np.full((Pn, Lm), -1, dtype=np.int64)
        r = 0
        for c in cands:
            cm[r:r + c.shape[0], :c.shape[1]] = c
            r += c.shape[0]
        px = np.concatenate(pxs)
        py = np.concatenate(pys)
        fr = fragments(params, cam, px, py, torch.from_numpy(cm), margins)
        pyt, pxt = torch.from_numpy(py), torch.from_numpy(px)
        vis_p = None if vis_t is None else vis_t[pyt, pxt]
        col = shade(fr["X"], fr["A"], fr["ray_d"], envp, Xind=fr["Xind"], vis=vis_p)
        rgba.index_put_((pyt, pxt), col)
        Xb.index_put_((pyt, pxt), fr["X"])
        Ab.index_put_((pyt, pxt), fr["A"])
        Zb.index_put_((pyt, pxt), fr["Z"])
        if fr["Xind"] is not None:
            Ib.index_put_((pyt, pxt), fr["Xind"])
        Tb.index_put_((pyt, pxt), fr["T"])
        n_eval[pyt, pxt] = fr["n_eval"]
        n_con[pyt, pxt] = fr["n_contrib"]
        last[pyt, pxt] = fr["last"]
        covered[pyt, pxt] = True
        if margins is not None:
            m = masks_and_alt(fr, envp, vis_p, col)
            amb[pyt, pxt] = m["ambiguous"]
            gamb[pyt, pxt] = m["grad_ambiguous"]
            for k in ("rgba", "X", "A", "Z", "T", "last"):
                alt[k][pyt, pxt] = m["alt"][k]
            alt["mask"][pyt, pxt] = m["alt_mask"]

    chunk, size = [], 0
    for tl in tile_list:
        L = brute_list.size if brute else int(kl["tile_ranges"][tl][1] - kl["tile_ranges"][tl][0])
        ent = K.TILE * K.TILE * max(L, 1)
        if chunk and size + ent > max_entries:
            run_chunk(chunk)
            chunk, size = [], 0
        chunk.append(tl)
        size += ent
    if chunk:
        run_chunk(chunk)
    return dict(rgba=rgba, X=Xb, A=Ab, Z=Zb, Xind=Ib, T=Tb, ambiguous=amb, grad_ambiguous=gamb, n_eval=n_eval,
                n_contrib=n_con, last=last, covered=covered, keys=kl, alt=alt)


def render_pixels(scene: dict, cam: dict, env: dict, px, py, *, keylist=None, params=None,
                  envp=None, margins=DEFAULT_MARGINS, vis=None) -> dict:
    """Render individual pixels (px, py) from their tiles' lists: the sampled
    check used at sizes where a whole image would take too long."""
    kl = keylist if keylist is not None else K.build_keys(scene, cam)
    params = params if params is not None else to_params(scene)
    envp = envp if envp is not None else env_params(env)
    tiles_x = kl["view"]["tiles_x"]
    px = np.asarray(px, dtype=np.int64)
    py = np.asarray(py, dtype=np.int64)
    cands = [tile_candidates(kl, (y // K.TILE) * tiles_x + (x // K.TILE)) for x, y in zip(px, py)]
    Lm = max(1, max(c.size for c in cands))
    cm = np.full((px.size, Lm), -1, dtype=np.int64)
    for i, c in enumerate(cands):
        cm[i, :c.size] = c
    fr = fragments(params, cam, px, py, torch.from_numpy(cm), margins)
    vis_p = None if vis is None else torch.from_numpy(np.asarray(vis, dtype=np.float64)[np.asarray(py), np.asarray(px)])
    col = shade(fr["X"], fr["A"], fr["ray_d"], envp, Xind=fr["Xind"], vis=vis_p)
    out = dict(rgba=col, X=fr["X"], A=fr["A"], Z=fr["Z"], T=fr["T"], n_eval=fr["n_eval"],
               n_contrib=fr["n_contrib"], last=fr["last"])
    if margins is not None:
        out.update(masks_and_alt(fr, envp, vis_p, col))
    return out


def masks_and_alt(fr: dict, envp: dict, vis_p, col: torch.Tensor) -> dict:
    """Per-pixel comparison masks of a fragments() result computed with margins.

    ambiguous       more than one decision within FP32 error of flipping (or
                    a shading decision there): no unique admissible result,
                    excluded from image comparisons;
    alt / alt_mask  exactly one such decision: the result with it flipped
                    (rgba, X, A, Z, T, last), the other admissible result;
    grad_ambiguous  any decision in its band, or a derivative kink: excluded
                    from gradient comparisons (a slope differs across them).
    """
    with torch.no_grad():
        X, A, d = fr["X"].detach(), fr["A"].detach(), fr["ray_d"]
        a = fr["alt"]
        Xind_a = a["Xind"].detach() if a["Xind"] is not None else None
        col_a = shade(a["X"].detach(), a["A"].detach(), d, envp, Xind=Xind_a, vis=vis_p).detach()
        single = fr["alt_mask"]
        amb = fr["ambiguous"] | shading_ambiguity(X, A, d) | (single & shading_ambiguity(a["X"], a["A"], d))
        single = single & ~amb
        # pixels without an alternative carry the definition's result there too
        sel = single[:, None]
        alt = dict(rgba=torch.where(sel, col_a, col.detach()), X=torch.where(sel, a["X"], X),
                   A=torch.where(single, a["A"], A), Z=torch.where(single, a["Z"], fr["Z"].detach()),
                   T=torch.where(single, a["T"], fr["T"].detach()), last=torch.where(single, a["last"], fr["last"]))
        gamb = amb | fr["decision_band"] | fr["kink"] | shading_kinks(X, A, d, envp)
    return dict(ambiguous=amb, alt_mask=single, alt=alt, grad_ambiguous=gamb)


def render_attributes_2dgs(scene: dict, cam: dict, env: dict, attrs: np.ndarray, **kw) -> dict:
    """Per-primitive-attribute 2DGS branch (one 8-vector per splat, no texture):
    the texture lookup is replaced by the splat's constant attribute.  Written
    separately from the texture path so that the 'constant texture equals
    per-splat attribute' invariant (Sec. 3.2, Sec. 4.1 two-stage training)
    compares two independent code paths."""
    W, H = int(cam["W"]), int(cam["H"])
    params = to_params(dict(scene, texels=np.zeros((len(scene["opacity"]), 1, 1, 8))))
    envp = env_params(env)
    kl = K.build_keys(scene, cam)
    tiles_x = kl["view"]["tiles_x"]
    attr = torch.from_numpy(np.asarray(attrs, dtype=np.float64))
    _, _, origin = camera_tensors(cam)
    tu_all, tv_all, n_all = rotation_columns(params["quats"])
    out = torch.zeros(H, W, 4, dtype=F64)
    for y in range(H):
        xs = np.arange(W)
        ys = np.full(W, y)
        d = pixel_rays(cam, xs, ys)
        for xi in range(W):
            tl = (y // K.TILE) * tiles_x + (xi // K.TILE)
            Tt = 1.0
            Xp = torch.zeros(8, dtype=F64)
            Ap = 0.0
            for k in tile_candidates(kl, tl):
                p, n = params["means"][k], n_all[k]
                den = float(d[xi] @ n)
                if abs(den) <= 1e-12 * float(torch.linalg.vector_norm(d[xi])):
                    continue
                num = float((p - origin) @ n)
                tau = num / den
                if tau <= NEAR:
                    continue
                rel = tau * d[xi] - (p - origin)
                u = float(rel @ tu_all[k]) / float(params["scales"][k, 0])
                v = float(rel @ tv_all[k]) / float(params["scales"][k, 1])
                if not (abs(u) <= 3.0 and abs(v) <= 3.0):
                    continue
                al = min(ALPHA_MAX, float(params["opacity"][k]) * math.exp(-(u * u + v * v) / 2.0))
                if al < ALPHA_MIN:
                    continue
                nf = -n if num > 0 else n
                nt = attr[k, 5:8]
                nw = nt[0] * tu_all[k] + nt[1] * tv_all[k] + nt[2] * nf
                xv = torch.cat([attr[k, 0:5], nw])
                Xp = Xp + al * Tt * xv
                Ap = Ap + al * Tt
                Tt = Tt * (1.0 - al)
                if Tt < T_MIN:
                    break
            out[y, xi, :] = shade(Xp[None], torch.tensor([Ap], dtype=F64), d[xi:xi + 1], envp)[0]
    return dict(rgba=out)
