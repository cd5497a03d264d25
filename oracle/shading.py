"""FP64 deferred physically based shading of the G-buffer (TEST INFRASTRUCTURE).

Follows Sec. 3.5 "Physically-Based Shading" (Eq. 10-12) with the readings
this renderer fixes where the paper defers to nvdiffrec:

  colour = A * L_o(Lam/A, M/A, R/A, N/|N|)  (background 0, colour 0 if A < 1e-7)
  L_o    = L_d + L_s                                              (Eq. 10)
  L_d    = Lam/pi * (1 - M) * E(N)        E = irradiance cube      (Eq. 11)
  L_s    = (F0 * LUT_A + LUT_B) * C_spec(w_r, lod = R * (levels-1))  (Eq. 12, V = 1, L_ind = 0)
  F0     = 0.04 * (1 - M) + Lam * M
  w_o    = -(pixel ray direction) normalised, NdotV = clamp(N.w_o, 1e-4, 1),
  w_r    = 2 (N.w_o) N - w_o

Cube maps are [6, R, R, 3] (face, row t, column s, channel), faces +x,-x,+y,
-y,+z,-z selected by the major axis (ties x > y > z) with the OpenGL/CUDA
face coordinates; texel centres, bilinear, clamp-to-edge inside the face.
The specular cube is a mip chain filtered trilinearly; the BRDF table is
[R_rough, R_NdotV, 2] sampled bilinearly at texel centres, clamp-to-edge.

Parity: pinned by the constant-radiance closed form and the analytic SH
irradiance comparison in tests/test_oracle_shading.py; the paper's own LUT,
mip filtering and environment maps are not available (parity unpinned for
those contents, which are inputs here).
"""
from __future__ import annotations

import math

import torch

A_MIN = float(torch.tensor(1e-7, dtype=torch.float32))
NDOTV_MIN = float(torch.tensor(1e-4, dtype=torch.float32))


def cube_face_coords(d: torch.Tensor):
    """Direction [...,3] -> (face index, s, t) on the cube, major axis ties
    resolved x > y > z.  Returns face (long), s, t in [0,1] and |ma|."""
    x, y, z = d[..., 0], d[..., 1], d[..., 2]
    ax, ay, az = x.abs(), y.abs(), z.abs()
    use_x = (ax >= ay) & (ax >= az)
    use_y = (~use_x) & (ay >= az)
    use_z = (~use_x) & (~use_y)
    face = torch.where(use_x, torch.where(x >= 0, 0, 1),
                       torch.where(use_y, torch.where(y >= 0, 2, 3), torch.where(z >= 0, 4, 5)))
    # (sc, tc, ma) per face:
    #  +x (-z,-y,x)  -x (z,-y,x)  +y (x,z,y)  -y (x,-z,y)  +z (x,-y,z)  -z (-x,-y,z)
    sc = torch.stack([-z, z, x, x, x, -x], -1)
    tc = torch.stack([-y, -y, z, -z, -y, -y], -1)
    ma = torch.stack([ax, ax, ay, ay, az, az], -1)
    fi = face.unsqueeze(-1)
    sc = torch.gather(sc, -1, fi).squeeze(-1)
    tc = torch.gather(tc, -1, fi).squeeze(-1)
    ma = torch.gather(ma, -1, fi).squeeze(-1)
    s = (sc / ma + 1.0) * 0.5
    t = (tc / ma + 1.0) * 0.5
    return face, s, t, ma


def bilinear_2d(img: torch.Tensor, x: torch.Tensor, y: torch.Tensor, lead_index=None):
    """Bilinear filter at continuous texel coordinates of texel-centre grids.

    ``img`` is [..., rows, cols, C]; (x, y) are in texel units where texel
    (row j, col i) has its centre at (i + 0.5, j + 0.5) / size, i.e. callers
    pass x = s * cols - 0.5.  Indices clamp to the edge of ``img``.
    ``lead_index`` (long, same shape as x) selects the leading index (face or
    splat) of a 4-D ``img``.
    """
    rows, cols = img.shape[-3], img.shape[-2]
    i0f = torch.floor(x)
    j0f = torch.floor(y)
    fx = (x - i0f).unsqueeze(-1)
    fy = (y - j0f).unsqueeze(-1)
    i0 = i0f.long()
    j0 = j0f.long()
    ia = i0.clamp(0, cols - 1)
    ib = (i0 + 1).clamp(0, cols - 1)
    ja = j0.clamp(0, rows - 1)
    jb = (j0 + 1).clamp(0, rows - 1)
    if lead_index is None:
        g = lambda j, i: img[j, i]  # noqa: E731
    else:
        g = lambda j, i: img[lead_index, j, i]  # noqa: E731
    top = (1.0 - fx) * g(ja, ia) + fx * g(ja, ib)
    bot = (1.0 - fx) * g(jb, ia) + fx * g(jb, ib)
    return (1.0 - fy) * top + fy * bot


def cube_sample(cube: torch.Tensor, d: torch.Tensor):
    """Bilinear sample of a [6,R,R,C] cube at directions d [...,3]."""
    face, s, t, _ = cube_face_coords(d)
    R = cube.shape[1]
    return bilinear_2d(cube, s * R - 0.5, t * R - 0.5, lead_index=face)


def cube_sample_lod(mips, d: torch.Tensor, lod: torch.Tensor):
    """Trilinear sample of a mip chain (list of [6,R_l,R_l,C]) at ``lod``."""
    L = len(mips)
    if L == 1:
        return cube_sample(mips[0], d)
    lodc = lod.clamp(0.0, float(L - 1))
    l0 = torch.floor(lodc).clamp(max=L - 1)
    f = (lodc - l0).unsqueeze(-1)
    l0i = l0.long()
    l1i = (l0i + 1).clamp(max=L - 1)
    out = torch.zeros(d.shape[:-1] + (mips[0].shape[-1],), dtype=d.dtype)
    for lv in range(L):
        val = cube_sample(mips[lv], d)
        wgt = torch.where(l0i == lv, 1.0 - f.squeeze(-1), torch.zeros_like(f.squeeze(-1)))
        wgt = wgt + torch.where(l1i == lv, f.squeeze(-1), torch.zeros_like(f.squeeze(-1)))
        out = out + wgt.unsqueeze(-1) * val
    return out


def lut_sample(lut: torch.Tensor, ndotv: torch.Tensor, rough: torch.Tensor):
    """Bilinear sample of the split-sum table at (NdotV, roughness)."""
    R_r, R_n = lut.shape[0], lut.shape[1]
    return bilinear_2d(lut, ndotv * R_n - 0.5, rough * R_r - 0.5)


# Real spherical harmonics up to degree 2 (the convention of the 3DGS line):
# Y_0 = 1/(2 sqrt(pi)); degree 1: -c1 y, c1 z, -c1 x with c1 = sqrt(3/(4 pi));
# degree 2: c2 xy, -c2 yz, c3 (2 z^2 - x^2 - y^2), -c2 xz, c4 (x^2 - y^2) with
# c2 = sqrt(15/(4 pi)), c3 = sqrt(5/(16 pi)), c4 = sqrt(15/(16 pi)).
SH_C0 = 0.5 / math.sqrt(math.pi)
SH_C1 = math.sqrt(3.0 / (4.0 * math.pi))
SH_C2 = math.sqrt(15.0 / (4.0 * math.pi))
SH_C3 = math.sqrt(5.0 / (16.0 * math.pi))
SH_C4 = math.sqrt(15.0 / (16.0 * math.pi))


def sh_basis(w: torch.Tensor, K: int) -> torch.Tensor:
    """[..., 3] unit directions -> [..., K] basis values, K in {1, 4, 9}."""
    x, y, z = w[..., 0], w[..., 1], w[..., 2]
    cols = [torch.full_like(x, SH_C0)]
    if K > 1:
        cols += [-SH_C1 * y, SH_C1 * z, -SH_C1 * x]
    if K > 4:
        cols += [SH_C2 * x * y, -SH_C2 * y * z, SH_C3 * (2.0 * z * z - x * x - y * y), -SH_C2 * x * z,
                 SH_C4 * (x * x - y * y)]
    return torch.stack(cols, -1)


def shade(X: torch.Tensor, A: torch.Tensor, ray_d: torch.Tensor, env: dict, Xind=None, vis=None):
    """Deferred shading of G-buffer pixels.

    X [P,8] blended (albedo RGB, metallic, roughness, normal xyz); A [P] the
    blended coverage; ray_d [P,3] world-space pixel ray directions; env holds
    torch tensors 'spec' (list of mips), 'irr', 'lut'.  With Xind [P,3] (the
    blended indirect light) and vis [P] (visibility V in [0, 1]) the specular
    light is V C_spec + (1 - V) Xind / A (Eq. 12 with L_ind).  Returns RGBA [P,4].
    """
    P = X.shape[0]
    ok = A >= A_MIN
    A_s = torch.where(ok, A, torch.ones_like(A))
    lam = X[:, 0:3] / A_s[:, None]
    met = X[:, 3] / A_s
    rough = X[:, 4] / A_s
    N = X[:, 5:8]
    wo = -ray_d / torch.linalg.vector_norm(ray_d, dim=-1, keepdim=True)
    nlen = torch.linalg.vector_norm(N, dim=-1, keepdim=True)
    nz = nlen >= 1e-12
    Nh = torch.where(nz, N / torch.where(nz, nlen, torch.ones_like(nlen)), wo)
    nv = (Nh * wo).sum(-1)
    ndotv = nv.clamp(NDOTV_MIN, 1.0)
    wr = 2.0 * nv[:, None] * Nh - wo
    f0 = 0.04 * (1.0 - met[:, None]) + lam * met[:, None]
    rc = rough.clamp(0.0, 1.0)
    lt = lut_sample(env["lut"], ndotv, rc)
    L = len(env["spec"])
    spec = cube_sample_lod(env["spec"], wr, rc * float(L - 1))
    irr = cube_sample(env["irr"], Nh)
    if Xind is not None:
        v = (torch.ones_like(A) if vis is None else vis)[:, None]
        spec = v * spec + (1.0 - v) * Xind / A_s[:, None]
    Ls = (f0 * lt[:, 0:1] + lt[:, 1:2]) * spec
    Ld = lam / math.pi * (1.0 - met[:, None]) * irr
    col = A_s[:, None] * (Ld + Ls)
    col = torch.where(ok[:, None], col, torch.zeros_like(col))
    return torch.cat([col, A[:, None]], -1).reshape(P, 4)


def normal_conditioning(X: torch.Tensor, A: torch.Tensor) -> torch.Tensor:
    """A / |N| (at least 1): how much the blended normal's direction amplifies
    rounding errors of its layers.  Layers whose normals partly cancel leave a
    short N whose direction an FP32 sum knows to fewer digits, so the margins
    of the shading's discrete decisions scale with it."""
    nlen = torch.linalg.vector_norm(X[:, 5:8], dim=-1)
    return torch.clamp(A / nlen.clamp_min(1e-30), min=1.0)


def shading_kinks(X: torch.Tensor, A: torch.Tensor, ray_d: torch.Tensor, env: dict, m_lut=2e-4, m_cube=2e-4,
                  m_clamp=1e-5):
    """Pixels whose shading gradient sits on a kink within FP32 error: a
    bilinear cell boundary of the BRDF table (N.w_o, roughness), of the
    specular cube (w_r, each sampled level) or of the irradiance cube (N),
    a mip-level boundary, or the N.w_o / roughness clamps.  Values are
    continuous there but derivatives jump, so FP32 and FP64 gradients may
    legitimately differ at such pixels."""
    with torch.no_grad():
        ok = A >= A_MIN
        A_s = torch.where(ok, A, torch.ones_like(A))
        rough = X[:, 4] / A_s
        N = X[:, 5:8]
        cond = normal_conditioning(X, A)
        m_lut, m_cube = m_lut * cond, m_cube * cond
        wo = -ray_d / torch.linalg.vector_norm(ray_d, dim=-1, keepdim=True)
        Nh = N / torch.linalg.vector_norm(N, dim=-1, keepdim=True).clamp_min(1e-300)
        nv = (Nh * wo).sum(-1)
        wr = 2.0 * nv[:, None] * Nh - wo
        rc = rough.clamp(0.0, 1.0)
        ndv = nv.clamp(NDOTV_MIN, 1.0)

        def near_kink(coord, size, m):
            fr = coord - torch.floor(coord)
            return ((fr <= m) | (fr >= 1.0 - m)) & (coord >= -m) & (coord <= size - 1 + m)

        Rl = env["lut"].shape[0]
        k = near_kink(ndv * Rl - 0.5, Rl, m_lut) | near_kink(rc * Rl - 0.5, Rl, m_lut)
        k |= ((nv - NDOTV_MIN).abs() <= m_clamp) | (rough.abs() <= m_clamp) | ((rough - 1.0).abs() <= m_clamp)
        L = len(env["spec"])
        _, s, t, _ = cube_face_coords(wr)
        for lv in range(L):
            R = env["spec"][lv].shape[1]
            k |= near_kink(s * R - 0.5, R, m_cube) | near_kink(t * R - 0.5, R, m_cube)
        if L > 1:
            lod = rc * float(L - 1)
            k |= near_kink(lod, L, m_cube)
        _, s, t, _ = cube_face_coords(Nh)
        R = env["irr"].shape[1]
        k |= near_kink(s * R - 0.5, R, m_cube) | near_kink(t * R - 0.5, R, m_cube)
    return k & ok


def shading_ambiguity(X: torch.Tensor, A: torch.Tensor, ray_d: torch.Tensor, m_face=3e-5,
                      m_small=1e-6):
    """Pixels whose shading takes a discrete decision within a hair of its
    switching point (cube face choice of w_r or N, the |N| fallback, the
    A < 1e-7 test), where FP32 and FP64 may legitimately differ."""
    with torch.no_grad():
        wo = -ray_d / torch.linalg.vector_norm(ray_d, dim=-1, keepdim=True)
        N = X[:, 5:8]
        nlen = torch.linalg.vector_norm(N, dim=-1)
        Nh = N / nlen.clamp_min(1e-300)[:, None]
        nv = (Nh * wo).sum(-1)
        wr = 2.0 * nv[:, None] * Nh - wo

        m_eff = m_face * normal_conditioning(X, A)

        def face_tie(d):
            a = d.abs().sort(-1, descending=True).values
            return (a[:, 0] - a[:, 1]) <= m_eff * a[:, 0]

        shaded = A >= A_MIN
        amb = shaded & (face_tie(wr) | face_tie(Nh) | (nlen < 1e-6))
        amb |= (A - A_MIN).abs() <= 1e-3 * A_MIN
    return amb
