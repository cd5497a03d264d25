"""Synthetic scenes shaped like object-centric reflective captures.

The paper evaluates on Shiny Blender / Glossy Synthetic / Ref-Real captures
(object in the middle, orbital cameras, ~800x800 renders).  Those datasets are
not available, so these seeded generators stand in for them.  The recipes are
the five workload configurations of the renderer:

  0  256 splats on a unit sphere, 4x4 texels, one 128x128 view (parity case)
  1  200k splats (160k sphere + 40k in a box), 8x8 texels, 100 views at 800x800
  2  500k sphere splats, 16x16 texels, 1920x1080, 6-level 128 cube
  3  serving: 200k / 500k / 1M scenes, 8x8 texels, mixed resolutions
  4  3M splats in a 10^3 box (60% on 32 spheres, 40% uniform), 1600x1064

Texel channel order (8 channels, one texel contiguous):
  0..2 albedo RGB, 3 metallic, 4 roughness, 5..7 tangent-space normal xyz.
Texel array layout: texels[k, row, col, c] with ``row`` along the splat's
v axis (texture t) and ``col`` along u (texture s).

Quaternions are (w, x, y, z); scales are linear (s_u, s_v); opacity is in
(0, 1).  Cameras are pinhole with OpenCV axes (x right, y down, z forward),
``R`` world->camera (row-major) and ``t`` world->camera translation.
"""
from __future__ import annotations

import functools
import math

import numpy as np
from scipy.spatial.transform import Rotation
from scipy.special import sph_harm_y

CONFIGS = {
    0: dict(n=256, box_frac=0.0, T=4, W=128, H=128, seed=0, cube_res=32, cube_levels=1,
            irr_res=8, n_cams=1, cam_radius=4.0),
    1: dict(n=200_000, box_frac=0.2, T=8, W=800, H=800, seed=1, cube_res=32, cube_levels=1,
            irr_res=8, n_cams=100, cam_radius=4.0),
    2: dict(n=500_000, box_frac=0.0, T=16, W=1920, H=1080, seed=2, cube_res=128, cube_levels=6,
            irr_res=16, n_cams=10, cam_radius=4.0),
    4: dict(n=3_000_000, box_frac=None, T=8, W=1600, H=1064, seed=4, cube_res=32, cube_levels=1,
            irr_res=8, n_cams=4, cam_radius=12.0),
}

LOG_SCALE_MEAN = math.log(0.05)
LOG_SCALE_SD = 0.3


def scene_config(cfg: int) -> dict:
    return dict(CONFIGS[cfg])


# ----------------------------------------------------------------------------
# orientation helpers (input construction only)
# ----------------------------------------------------------------------------

def frames_to_quats(tu: np.ndarray, tv: np.ndarray, n: np.ndarray) -> np.ndarray:
    """Quaternions (w,x,y,z) of the rotations whose columns are (tu, tv, n)."""
    mats = np.stack([tu, tv, n], axis=-1)  # columns
    xyzw = Rotation.from_matrix(mats).as_quat()
    return np.concatenate([xyzw[:, 3:4], xyzw[:, :3]], axis=1)


def random_unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniformly random rotations as unit quaternions (w,x,y,z)."""
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _tangent_frames(normals: np.ndarray, twist: np.ndarray):
    """Tangent frames with third axis ``normals`` and an in-plane twist."""
    ref = np.zeros_like(normals)
    use_x = np.abs(normals[:, 2]) > 0.9
    ref[~use_x, 2] = 1.0
    ref[use_x, 0] = 1.0
    a = np.cross(normals, ref)
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b = np.cross(normals, a)
    c, s = np.cos(twist)[:, None], np.sin(twist)[:, None]
    tu = c * a + s * b
    tv = np.cross(normals, tu)
    return tu, tv


def _sphere_splats(rng, n):
    """Centres uniform on the unit sphere + N(0, 0.02^2) noise, tangent frames."""
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    means = d + rng.normal(scale=0.02, size=(n, 3))
    twist = rng.uniform(0.0, 2.0 * math.pi, size=n)
    tu, tv = _tangent_frames(d, twist)
    quats = frames_to_quats(tu, tv, d)
    return means, quats


def _texels(rng, n, T):
    """Albedo U[0,1]^3, metallic U[0,1], roughness U[0.05,1], tangent normals
    normalise(N(0,0.2), N(0,0.2), 1)."""
    tex = np.empty((n, T, T, 8), dtype=np.float32)
    tex[..., 0:3] = rng.uniform(0.0, 1.0, size=(n, T, T, 3))
    tex[..., 3] = rng.uniform(0.0, 1.0, size=(n, T, T))
    tex[..., 4] = rng.uniform(0.05, 1.0, size=(n, T, T))
    nxy = rng.normal(scale=0.2, size=(n, T, T, 2))
    nrm = np.sqrt(nxy[..., 0] ** 2 + nxy[..., 1] ** 2 + 1.0)
    tex[..., 5] = nxy[..., 0] / nrm
    tex[..., 6] = nxy[..., 1] / nrm
    tex[..., 7] = 1.0 / nrm
    return tex


def texels_torch(n: int, T: int, seed: int, device="cuda"):
    """The texel distributions of :func:`_texels` drawn with torch's seeded
    generator on ``device`` (for multi-GB scenes; a different random stream
    than the numpy version)."""
    import torch
    g = torch.Generator(device=device).manual_seed(seed)
    tex = torch.empty(n, T, T, 8, dtype=torch.float32, device=device)
    tex[..., 0:4].uniform_(0.0, 1.0, generator=g)
    tex[..., 4].uniform_(0.05, 1.0, generator=g)
    nxy = torch.empty(n, T, T, 2, dtype=torch.float32, device=device).normal_(0.0, 0.2, generator=g)
    nrm = torch.sqrt(nxy[..., 0] ** 2 + nxy[..., 1] ** 2 + 1.0)
    tex[..., 5] = nxy[..., 0] / nrm
    tex[..., 6] = nxy[..., 1] / nrm
    tex[..., 7] = 1.0 / nrm
    return tex


def _common_params(rng, n):
    scales = np.exp(rng.normal(LOG_SCALE_MEAN, LOG_SCALE_SD, size=(n, 2)))
    opacity = 1.0 / (1.0 + np.exp(-rng.normal(size=n)))
    return scales, opacity


def make_scene(cfg: int = 0, n: int | None = None, T: int | None = None,
               seed: int | None = None, with_texels: bool = True) -> dict:
    """Build the splat cloud of configuration ``cfg`` (optionally resized).

    cfg 0/2: all splats on the unit sphere.  cfg 1 (and 3): 80% sphere,
    20% uniform in [-1,1]^3 with uniformly random orientation.  cfg 4: 60% on
    32 random spheres (radius U[0.3,1.5]) inside [-5,5]^3, 40% uniform in the
    box with random orientation.
    """
    c = scene_config(cfg if cfg in CONFIGS else 1)
    n = c["n"] if n is None else int(n)
    T = c["T"] if T is None else int(T)
    seed = c["seed"] if seed is None else int(seed)
    rng = np.random.default_rng(seed)
    if cfg == 4:
        n_surf = int(round(0.6 * n))
        centres = rng.uniform(-3.5, 3.5, size=(32, 3))
        radii = rng.uniform(0.3, 1.5, size=32)
        which = rng.integers(0, 32, size=n_surf)
        d = rng.normal(size=(n_surf, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        m_s = centres[which] + radii[which, None] * d
        tw = rng.uniform(0.0, 2.0 * math.pi, size=n_surf)
        tu, tv = _tangent_frames(d, tw)
        q_s = frames_to_quats(tu, tv, d)
        n_box = n - n_surf
        m_b = rng.uniform(-5.0, 5.0, size=(n_box, 3))
        q_b = random_unit_quats(rng, n_box)
        means = np.concatenate([m_s, m_b])
        quats = np.concatenate([q_s, q_b])
    else:
        box_frac = c["box_frac"] or 0.0
        n_box = int(round(box_frac * n))
        n_sph = n - n_box
        m_s, q_s = _sphere_splats(rng, n_sph)
        m_b = rng.uniform(-1.0, 1.0, size=(n_box, 3))
        q_b = random_unit_quats(rng, n_box)
        means = np.concatenate([m_s, m_b])
        quats = np.concatenate([q_s, q_b])
    scales, opacity = _common_params(rng, n)
    scene = dict(
        means=np.ascontiguousarray(means, dtype=np.float32),
        quats=np.ascontiguousarray(quats, dtype=np.float32),
        scales=np.ascontiguousarray(scales, dtype=np.float32),
        opacity=np.ascontiguousarray(opacity, dtype=np.float32),
        T=T,
    )
    if with_texels:
        scene["texels"] = _texels(rng, n, T)
    return scene


def slice_scene(scene: dict, idx) -> dict:
    """Sub-scene holding splats ``idx`` (e.g. ``slice(0, 1000)``)."""
    out = {k: (v[idx].copy() if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
    return out


# ----------------------------------------------------------------------------
# cameras
# ----------------------------------------------------------------------------

def look_at_camera(eye, W: int, H: int, fov_deg: float = 40.0, target=(0.0, 0.0, 0.0)) -> dict:
    """Pinhole camera at ``eye`` looking at ``target``.  Vertical fov, square
    pixels: fx = fy = (H/2)/tan(fov/2), cx = W/2, cy = H/2.  World up is +z,
    falling back to +y when the view direction is within ~8 deg of it."""
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    up = np.array([0.0, 0.0, 1.0])
    if abs(f @ up) > 0.99:
        up = np.array([0.0, 1.0, 0.0])
    right = np.cross(f, up)
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    R = np.stack([right, down, f])  # rows: camera axes in world coordinates
    t = -R @ eye
    foc = (H / 2.0) / math.tan(math.radians(fov_deg) / 2.0)
    return dict(R=R.astype(np.float32), t=t.astype(np.float32), fx=np.float32(foc),
                fy=np.float32(foc), cx=np.float32(W / 2.0), cy=np.float32(H / 2.0),
                W=int(W), H=int(H))


def fibonacci_cameras(n: int, radius: float, W: int, H: int, fov_deg: float = 40.0):
    """``n`` cameras on a Fibonacci sphere of ``radius``, looking at the origin."""
    cams = []
    golden = math.pi * (3.0 - math.sqrt(5.0))
    for i in range(n):
        z = 1.0 - 2.0 * (i + 0.5) / n
        r = math.sqrt(max(0.0, 1.0 - z * z))
        phi = golden * i
        eye = radius * np.array([r * math.cos(phi), r * math.sin(phi), z])
        cams.append(look_at_camera(eye, W, H, fov_deg))
    return cams


def random_sphere_cameras(rng: np.random.Generator, n: int, rmin: float, rmax: float,
                          resolutions, fov_deg: float = 40.0):
    """Cameras uniform on spheres of radius U[rmin, rmax], resolution drawn
    uniformly from ``resolutions`` [(W,H), ...]."""
    cams = []
    for _ in range(n):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        r = rng.uniform(rmin, rmax)
        W, H = resolutions[rng.integers(0, len(resolutions))]
        cams.append(look_at_camera(r * d, W, H, fov_deg))
    return cams


# ----------------------------------------------------------------------------
# environment light and BRDF table (data, precomputed on the host)
# ----------------------------------------------------------------------------

def cube_texel_dirs(res: int) -> np.ndarray:
    """Unit directions through the texel centres of a cube map [6,res,res,3].

    Face order +x, -x, +y, -y, +z, -z; within a face, texel (row j, col i)
    has face coordinates sc = 2(i+0.5)/res - 1, tc = 2(j+0.5)/res - 1 and the
    face axes of the usual OpenGL/CUDA cube convention:
      +x: (1, -tc, -sc)   -x: (-1, -tc, sc)   +y: (sc, 1, tc)
      -y: (sc, -1, -tc)   +z: (sc, -tc, 1)    -z: (-sc, -tc, -1)
    """
    c = (np.arange(res) + 0.5) / res * 2.0 - 1.0
    tc, sc = np.meshgrid(c, c, indexing="ij")
    one = np.ones_like(sc)
    faces = [
        np.stack([one, -tc, -sc], -1),
        np.stack([-one, -tc, sc], -1),
        np.stack([sc, one, tc], -1),
        np.stack([sc, -one, -tc], -1),
        np.stack([sc, -tc, one], -1),
        np.stack([-sc, -tc, -one], -1),
    ]
    d = np.stack(faces)
    return d / np.linalg.norm(d, axis=-1, keepdims=True)


def _real_sh(lmax: int, dirs: np.ndarray) -> np.ndarray:
    """Orthonormal real spherical harmonics up to degree lmax at unit dirs."""
    x, y, z = dirs[..., 0], dirs[..., 1], dirs[..., 2]
    theta = np.arccos(np.clip(z, -1.0, 1.0))
    phi = np.mod(np.arctan2(y, x), 2.0 * math.pi)
    out = []
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            if m < 0:
                v = math.sqrt(2.0) * (-1) ** m * np.imag(sph_harm_y(l, -m, theta, phi))
            elif m == 0:
                v = np.real(sph_harm_y(l, 0, theta, phi))
            else:
                v = math.sqrt(2.0) * (-1) ** m * np.real(sph_harm_y(l, m, theta, phi))
            out.append(v)
    return np.stack(out, -1)


# cosine-lobe convolution factors per SH degree (Ramamoorthi & Hanrahan 2001)
_COS_LOBE = [math.pi, 2.0 * math.pi / 3.0, math.pi / 4.0, 0.0, -math.pi / 24.0]


def sh_env_coeffs(seed: int, lmax: int = 4) -> np.ndarray:
    """Radiance SH coefficients [(lmax+1)^2, 3]: 0.5 ambient + N(0,(0.15/(l+1))^2)."""
    rng = np.random.default_rng(10_000 + seed)
    coeffs = []
    for l in range(lmax + 1):
        for _m in range(2 * l + 1):
            coeffs.append(rng.normal(scale=0.15 / (l + 1), size=3))
    c = np.array(coeffs)
    c[0] += 0.5 / _real_sh(0, np.array([[0.0, 0.0, 1.0]]))[0, 0]
    return c


def sh_radiance(coeffs: np.ndarray, dirs: np.ndarray) -> np.ndarray:
    lmax = int(round(math.sqrt(coeffs.shape[0]))) - 1
    return _real_sh(lmax, dirs) @ coeffs


def sh_irradiance(coeffs: np.ndarray, dirs: np.ndarray) -> np.ndarray:
    """Analytic irradiance E(n) = sum_l A_l sum_m c_lm Y_lm(n) of the SH radiance."""
    lmax = int(round(math.sqrt(coeffs.shape[0]))) - 1
    scale = np.concatenate([[_COS_LOBE[l]] * (2 * l + 1) for l in range(lmax + 1)])
    return _real_sh(lmax, dirs) @ (coeffs * scale[:, None])


def make_env(seed: int = 0, cube_res: int = 32, levels: int = 1, irr_res: int = 8,
             lut_res: int = 128) -> dict:
    """Environment light as data: specular mip chain (level 0 = SH radiance at
    texel centres, each next level a 2x2 box average), irradiance cube (the
    analytic cosine convolution of the same SH) and the split-sum BRDF table."""
    coeffs = sh_env_coeffs(seed)
    spec = [sh_radiance(coeffs, cube_texel_dirs(cube_res)).astype(np.float32)]
    for _ in range(1, levels):
        prev = spec[-1].astype(np.float64)
        r = prev.shape[1] // 2
        nxt = prev.reshape(6, r, 2, r, 2, 3).mean(axis=(2, 4))
        spec.append(nxt.astype(np.float32))
    irr = sh_irradiance(coeffs, cube_texel_dirs(irr_res)).astype(np.float32)
    return dict(spec=spec, irr=irr, lut=brdf_lut(lut_res), sh=coeffs)


def constant_env(c, cube_res=8, levels=1, irr_res=4, lut=(1.0, 0.0), lut_res=8) -> dict:
    """Constant radiance ``c`` (RGB): irradiance pi*c, LUT constant (A0, B0)."""
    c = np.asarray(c, dtype=np.float32).reshape(3)
    spec = []
    r = cube_res
    for _ in range(levels):
        spec.append(np.broadcast_to(c, (6, r, r, 3)).astype(np.float32).copy())
        r = max(1, r // 2)
    irr = np.broadcast_to(np.float32(math.pi) * c, (6, irr_res, irr_res, 3)).astype(np.float32).copy()
    lt = np.empty((lut_res, lut_res, 2), dtype=np.float32)
    lt[..., 0] = lut[0]
    lt[..., 1] = lut[1]
    return dict(spec=spec, irr=irr, lut=lt)


def _radical_inverse2(i: np.ndarray) -> np.ndarray:
    i = i.astype(np.uint32)
    i = ((i << 16) | (i >> 16)).astype(np.uint32)
    i = (((i & 0x55555555) << 1) | ((i & 0xAAAAAAAA) >> 1)).astype(np.uint32)
    i = (((i & 0x33333333) << 2) | ((i & 0xCCCCCCCC) >> 2)).astype(np.uint32)
    i = (((i & 0x0F0F0F0F) << 4) | ((i & 0xF0F0F0F0) >> 4)).astype(np.uint32)
    i = (((i & 0x00FF00FF) << 8) | ((i & 0xFF00FF00) >> 8)).astype(np.uint32)
    return i.astype(np.float64) / 4294967296.0


@functools.lru_cache(maxsize=8)
def brdf_lut(res: int = 128, nsamp: int = 512) -> np.ndarray:
    """Split-sum GGX/Smith BRDF table [res_rough, res_NdotV, 2] (Karis 2013):
    column i <-> NdotV = (i+0.5)/res, row j <-> roughness = (j+0.5)/res,
    channels (scale A, bias B) with F0*A + B the pre-integrated reflectance.
    Importance-sampled GGX with alpha = roughness^2, Smith-Schlick k = alpha/2,
    Hammersley points."""
    nov = (np.arange(res) + 0.5) / res
    rough = (np.arange(res) + 0.5) / res
    NV, RG = np.meshgrid(nov, rough)  # [row=rough, col=nov]
    i = np.arange(nsamp)
    xi1 = i / nsamp
    xi2 = _radical_inverse2(i)
    a = (RG ** 2)[..., None]
    phi = 2.0 * math.pi * xi1
    cos_t = np.sqrt((1.0 - xi2) / (1.0 + (a * a - 1.0) * xi2))
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    hx, hy, hz = sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t
    vx = np.sqrt(1.0 - NV ** 2)[..., None]
    vz = NV[..., None]
    voh = vx * hx + vz * hz
    lz = 2.0 * voh * hz - vz
    nol = np.clip(lz, 0.0, 1.0)
    noh = np.clip(hz, 0.0, 1.0)
    voh_c = np.clip(voh, 0.0, 1.0)
    k = a / 2.0
    g1v = vz / (vz * (1.0 - k) + k)
    g1l = nol / (nol * (1.0 - k) + k)
    gvis = g1v * g1l * voh_c / np.maximum(noh * vz, 1e-12)
    fc = (1.0 - voh_c) ** 5
    valid = lz > 0.0
    A = np.where(valid, (1.0 - fc) * gvis, 0.0).mean(-1)
    B = np.where(valid, fc * gvis, 0.0).mean(-1)
    return np.stack([A, B], -1).astype(np.float32)


def make_target(cam_index: int, W: int, H: int) -> np.ndarray:
    """Seeded U[0,1] RGBA target image [H, W, 4] (alpha target 1)."""
    rng = np.random.default_rng(1000 + cam_index)
    img = np.ones((H, W, 4), dtype=np.float32)
    img[..., :3] = rng.uniform(0.0, 1.0, size=(H, W, 3))
    return img
