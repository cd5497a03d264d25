// Deferred split-sum shading of one G-buffer pixel and its adjoint (FP32).
//
// TextureSplat Sec. 3.5.4 (Eq. 10-12) with V = 1 and no indirect term:
//   colour = A * (L_d + L_s) evaluated at the normalised buffers
//   Lam = X[0:3]/A, M = X[3]/A, R = X[4]/A, N = X[5:8]/|X[5:8]|
//   L_d = Lam/pi (1 - M) E(N)                       (irradiance cube)
//   L_s = (F0 LUT_A + LUT_B) C_spec(w_r, R (levels-1))  (trilinear mip chain)
//   F0 = 0.04 (1 - M) + Lam M,  w_o = -d/|d|,  w_r = 2 (N.w_o) N - w_o
//   colour = 0 when A < 1e-7; alpha channel = A.
// Cube faces +x,-x,+y,-y,+z,-z, major axis ties x > y > z, OpenGL face
// coordinates, texel centres, bilinear with clamp-to-edge in the face.
#pragma once
#include "ts_common.cuh"

namespace ts {

struct Bil {
  int ia, ib, ja, jb;
  float fx, fy;
};

__device__ __forceinline__ Bil bil_setup(float x, float y, int cols, int rows) {
  Bil b;
  float fi = floorf(x), fj = floorf(y);
  b.fx = x - fi;
  b.fy = y - fj;
  int i0 = (int)fi, j0 = (int)fj;
  b.ia = min(max(i0, 0), cols - 1);
  b.ib = min(max(i0 + 1, 0), cols - 1);
  b.ja = min(max(j0, 0), rows - 1);
  b.jb = min(max(j0 + 1, 0), rows - 1);
  return b;
}

struct CubeCoord {
  int face;
  float s, t;   // face coordinates in [0,1]
  float sc, tc, ma;
};

__device__ __forceinline__ CubeCoord cube_coord(float3 d) {
  CubeCoord c;
  float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
  if (ax >= ay && ax >= az) {
    c.face = d.x >= 0.f ? 0 : 1;
    c.ma = ax;
    c.sc = d.x >= 0.f ? -d.z : d.z;
    c.tc = -d.y;
  } else if (ay >= az) {
    c.face = d.y >= 0.f ? 2 : 3;
    c.ma = ay;
    c.sc = d.x;
    c.tc = d.y >= 0.f ? d.z : -d.z;
  } else {
    c.face = d.z >= 0.f ? 4 : 5;
    c.ma = az;
    c.sc = d.z >= 0.f ? d.x : -d.x;
    c.tc = -d.y;
  }
  c.s = (c.sc / c.ma + 1.f) * 0.5f;
  c.t = (c.tc / c.ma + 1.f) * 0.5f;
  return c;
}

// Bilinear sample of one cube face of resolution R; also returns d/dx, d/dy
// (per texel unit) when grad != nullptr.
__device__ __forceinline__ float3 cube_bilinear(const void* cube, int dtype, int R, const CubeCoord& c,
                                                Bil& b, float3* ddx, float3* ddy) {
  b = bil_setup(c.s * R - 0.5f, c.t * R - 0.5f, R, R);
  long long fb = (long long)c.face * R * R;
  float3 tAA = load_cube3(cube, dtype, fb + (long long)b.ja * R + b.ia);
  float3 tAB = load_cube3(cube, dtype, fb + (long long)b.ja * R + b.ib);
  float3 tBA = load_cube3(cube, dtype, fb + (long long)b.jb * R + b.ia);
  float3 tBB = load_cube3(cube, dtype, fb + (long long)b.jb * R + b.ib);
  float gx = 1.f - b.fx, gy = 1.f - b.fy;
  float3 top = make_float3(gx * tAA.x + b.fx * tAB.x, gx * tAA.y + b.fx * tAB.y, gx * tAA.z + b.fx * tAB.z);
  float3 bot = make_float3(gx * tBA.x + b.fx * tBB.x, gx * tBA.y + b.fx * tBB.y, gx * tBA.z + b.fx * tBB.z);
  if (ddx) {
    *ddx = make_float3(gy * (tAB.x - tAA.x) + b.fy * (tBB.x - tBA.x), gy * (tAB.y - tAA.y) + b.fy * (tBB.y - tBA.y),
                       gy * (tAB.z - tAA.z) + b.fy * (tBB.z - tBA.z));
    *ddy = make_float3(bot.x - top.x, bot.y - top.y, bot.z - top.z);
  }
  return make_float3(gy * top.x + b.fy * bot.x, gy * top.y + b.fy * bot.y, gy * top.z + b.fy * bot.z);
}

// d(s,t) of a cube lookup -> d(direction).
__device__ __forceinline__ float3 cube_coord_grad(const CubeCoord& c, float gs, float gt) {
  float ima = 1.f / c.ma;
  float gsc = 0.5f * gs * ima, gtc = 0.5f * gt * ima;
  float gma = -0.5f * (gs * c.sc + gt * c.tc) * ima * ima;
  switch (c.face) {
    case 0: return make_float3(gma, -gtc, -gsc);
    case 1: return make_float3(-gma, -gtc, gsc);
    case 2: return make_float3(gsc, gma, gtc);
    case 3: return make_float3(gsc, -gma, -gtc);
    case 4: return make_float3(gsc, -gtc, gma);
    default: return make_float3(-gsc, -gtc, -gma);
  }
}

__device__ __forceinline__ float2 lut_bilinear(const float* lut, int R, float ndv, float rough, Bil& b,
                                               float2* ddx, float2* ddy) {
  b = bil_setup(ndv * R - 0.5f, rough * R - 0.5f, R, R);
  const float2* L = reinterpret_cast<const float2*>(lut);
  float2 tAA = __ldg(L + b.ja * R + b.ia), tAB = __ldg(L + b.ja * R + b.ib);
  float2 tBA = __ldg(L + b.jb * R + b.ia), tBB = __ldg(L + b.jb * R + b.ib);
  float gx = 1.f - b.fx, gy = 1.f - b.fy;
  float2 top = make_float2(gx * tAA.x + b.fx * tAB.x, gx * tAA.y + b.fx * tAB.y);
  float2 bot = make_float2(gx * tBA.x + b.fx * tBB.x, gx * tBA.y + b.fx * tBB.y);
  if (ddx) {
    *ddx = make_float2(gy * (tAB.x - tAA.x) + b.fy * (tBB.x - tBA.x), gy * (tAB.y - tAA.y) + b.fy * (tBB.y - tBA.y));
    *ddy = make_float2(bot.x - top.x, bot.y - top.y);
  }
  return make_float2(gy * top.x + b.fy * bot.x, gy * top.y + b.fy * bot.y);
}

struct ShadeState {
  float lam[3], met, rough, rc;
  float3 N, Nh, wo, wr;
  float nlen, nv, ndv;
  float F0[3];
  float2 lt;
  float3 spec, irr;
  float lod, f;
  int l0, l1;
  bool ok, nz;
  // lookups kept for the adjoint (filled when shade_pixel is asked for them)
  CubeCoord cr, cn;
  Bil b0, b1, bi;
  float2 ldx, ldy;          // d LUT / d (NdotV, roughness) texel units
  float3 c0, c1;            // specular samples at levels l0, l1
  float3 dx0, dy0, dx1, dy1, idx, idy;  // their texel-unit derivatives
};

__device__ __forceinline__ float3 world_ray(const ViewDesc& V, float xp, float yp) {
  // d = R^T (x'/fx, y'/fy, 1)
  float a = xp / V.fx, b = yp / V.fy;
  return make_float3(V.R[0] * a + V.R[3] * b + V.R[6], V.R[1] * a + V.R[4] * b + V.R[7],
                     V.R[2] * a + V.R[5] * b + V.R[8]);
}

// ind (optional): the blended indirect light X_ind (3 channels, not yet
// divided by A) and vis the pixel's visibility V: the specular light becomes
// V C_spec + (1 - V) X_ind / A (Eq. 12 with L_ind).
template <bool GRAD = false>
__device__ __forceinline__ float4 shade_pixel(const EnvDesc& E, const float X[8], float A, float3 d,
                                              ShadeState* st, const float* ind = nullptr, float vis = 1.f) {
  ShadeState s;
  s.ok = A >= kAMin();
  if (!s.ok) {
    if (st) *st = s;
    return make_float4(0.f, 0.f, 0.f, A);
  }
  float iA = 1.f / A;
  s.lam[0] = X[0] * iA; s.lam[1] = X[1] * iA; s.lam[2] = X[2] * iA;
  s.met = X[3] * iA;
  s.rough = X[4] * iA;
  s.N = make_float3(X[5], X[6], X[7]);
  float idl = rsqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
  s.wo = make_float3(-d.x * idl, -d.y * idl, -d.z * idl);
  s.nlen = sqrtf(s.N.x * s.N.x + s.N.y * s.N.y + s.N.z * s.N.z);
  s.nz = s.nlen >= 1e-12f;
  if (s.nz) {
    float inl = 1.f / s.nlen;
    s.Nh = make_float3(s.N.x * inl, s.N.y * inl, s.N.z * inl);
  } else {
    s.Nh = s.wo;
  }
  s.nv = s.Nh.x * s.wo.x + s.Nh.y * s.wo.y + s.Nh.z * s.wo.z;
  s.ndv = fminf(fmaxf(s.nv, kNdotVMin()), 1.f);
  s.wr = make_float3(2.f * s.nv * s.Nh.x - s.wo.x, 2.f * s.nv * s.Nh.y - s.wo.y, 2.f * s.nv * s.Nh.z - s.wo.z);
#pragma unroll
  for (int c = 0; c < 3; ++c) s.F0[c] = 0.04f * (1.f - s.met) + s.lam[c] * s.met;
  s.rc = fminf(fmaxf(s.rough, 0.f), 1.f);
  Bil bl;
  s.lt = lut_bilinear(E.lut, E.lut_res, s.ndv, s.rc, bl, GRAD ? &s.ldx : nullptr, GRAD ? &s.ldy : nullptr);
  s.cr = cube_coord(s.wr);
  int L = E.levels;
  s.lod = s.rc * (float)(L - 1);
  float l0f = fminf(floorf(s.lod), (float)(L - 1));
  s.f = s.lod - l0f;
  s.l0 = (int)l0f;
  s.l1 = min(s.l0 + 1, L - 1);
  s.c0 = cube_bilinear(E.spec[s.l0], E.cube_dtype, E.spec_res[s.l0], s.cr, s.b0, GRAD ? &s.dx0 : nullptr,
                       GRAD ? &s.dy0 : nullptr);
  const float3 c0 = s.c0;
  if (L > 1) {
    s.c1 = cube_bilinear(E.spec[s.l1], E.cube_dtype, E.spec_res[s.l1], s.cr, s.b1, GRAD ? &s.dx1 : nullptr,
                         GRAD ? &s.dy1 : nullptr);
    const float3 c1 = s.c1;
    float g = 1.f - s.f;
    s.spec = make_float3(g * c0.x + s.f * c1.x, g * c0.y + s.f * c1.y, g * c0.z + s.f * c1.z);
  } else {
    s.spec = c0;
  }
  s.cn = cube_coord(s.Nh);
  s.irr = cube_bilinear(E.irr, E.cube_dtype, E.irr_res, s.cn, s.bi, GRAD ? &s.idx : nullptr, GRAD ? &s.idy : nullptr);
  const float inv_pi = 0.318309886183790672f;
  float spec3[3] = {s.spec.x, s.spec.y, s.spec.z};
  if (ind) {
#pragma unroll
    for (int c = 0; c < 3; ++c) spec3[c] = fmaf(vis, spec3[c], (1.f - vis) * ind[c] * iA);
  }
  float irr3[3] = {s.irr.x, s.irr.y, s.irr.z};
  float col[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float Ls = (s.F0[c] * s.lt.x + s.lt.y) * spec3[c];
    float Ld = s.lam[c] * inv_pi * (1.f - s.met) * irr3[c];
    col[c] = A * (Ld + Ls);
  }
  if (st) *st = s;
  return make_float4(col[0], col[1], col[2], A);
}

// What the environment maps receive from one pixel: gsp (3 channels) with
// bilinear weights at level l0 (times w0) and l1 (times w1, when levels > 1)
// of the specular chain, gir at the irradiance cube.
struct EnvGrad {
  bool ok;
  int l0, l1, face_r, face_n;
  Bil b0, b1, bi;
  float w0, w1;
  float3 gsp, gir;
};

// Adjoint of shade_pixel: given dL/drgba returns dL/dX (8) and dL/dA, and
// the environment-map gradient of the pixel in `eg` (scattered by the caller).
// With ind / vis as in shade_pixel, gind (3) receives dL/dX_ind.
__device__ __forceinline__ void shade_pixel_bwd(const EnvDesc& E, const float X[8], float A, float3 d,
                                                float4 g, float gX[8], float& gA, EnvGrad& eg,
                                                const float* ind = nullptr, float vis = 1.f,
                                                float* gind = nullptr) {
#pragma unroll
  for (int c = 0; c < 8; ++c) gX[c] = 0.f;
  ShadeState s;
  shade_pixel<true>(E, X, A, d, &s);
  gA = g.w;
  eg.ok = s.ok;
  if (gind) gind[0] = gind[1] = gind[2] = 0.f;
  if (!s.ok) return;
  const float inv_pi = 0.318309886183790672f;
  float gc[3] = {g.x, g.y, g.z};
  const float iAs = 1.f / A;
  float spec3[3] = {s.spec.x, s.spec.y, s.spec.z};  // the mixed specular light M
  if (ind) {
#pragma unroll
    for (int c = 0; c < 3; ++c) spec3[c] = fmaf(vis, spec3[c], (1.f - vis) * ind[c] * iAs);
  }
  float irr3[3] = {s.irr.x, s.irr.y, s.irr.z};
  float gLo[3], glam[3] = {0.f, 0.f, 0.f}, gmet = 0.f, gF0[3];
  float gspec3[3], girr3[3];
  float gLA = 0.f, gLB = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float Ls = (s.F0[c] * s.lt.x + s.lt.y) * spec3[c];
    float Ld = s.lam[c] * inv_pi * (1.f - s.met) * irr3[c];
    gA += gc[c] * (Ld + Ls);
    gLo[c] = A * gc[c];
    // L_d
    glam[c] += (1.f - s.met) * inv_pi * irr3[c] * gLo[c];
    gmet -= s.lam[c] * inv_pi * irr3[c] * gLo[c];
    girr3[c] = s.lam[c] * inv_pi * (1.f - s.met) * gLo[c];
    // L_s
    gF0[c] = s.lt.x * spec3[c] * gLo[c];
    gLA += s.F0[c] * spec3[c] * gLo[c];
    gLB += spec3[c] * gLo[c];
    gspec3[c] = (s.F0[c] * s.lt.x + s.lt.y) * gLo[c];  // dL/dM
    if (ind) {
      const float gi = (1.f - vis) * gspec3[c] * iAs;  // M = V C + (1 - V) X_ind / A
      gind[c] = gi;
      gA -= gi * ind[c] * iAs;
      gspec3[c] *= vis;  // -> dL/dC_spec
    }
    // F0
    glam[c] += s.met * gF0[c];
    gmet += (s.lam[c] - 0.04f) * gF0[c];
  }
  // LUT (not learnable): gradient to NdotV and roughness
  const float2 ldx = s.ldx, ldy = s.ldy;
  float gndv = (float)E.lut_res * (gLA * ldx.x + gLB * ldx.y);
  float grc = (float)E.lut_res * (gLA * ldy.x + gLB * ldy.y);
  // specular cube, trilinear
  const CubeCoord& cr = s.cr;
  int L = E.levels;
  float3 gwr = make_float3(0.f, 0.f, 0.f);
  float3 gsp = make_float3(gspec3[0], gspec3[1], gspec3[2]);
  {
    const Bil b0 = s.b0;
    const float3 dx0 = s.dx0, dy0 = s.dy0, c0 = s.c0;
    float R0 = (float)E.spec_res[s.l0];
    float w0 = (L > 1) ? (1.f - s.f) : 1.f;
    float gs = w0 * R0 * (gsp.x * dx0.x + gsp.y * dx0.y + gsp.z * dx0.z);
    float gt = w0 * R0 * (gsp.x * dy0.x + gsp.y * dy0.y + gsp.z * dy0.z);
    eg.l0 = s.l0;
    eg.l1 = s.l1;
    eg.face_r = cr.face;
    eg.b0 = b0;
    eg.b1 = b0;
    eg.w0 = w0;
    eg.w1 = 0.f;
    eg.gsp = gsp;
    if (L > 1) {
      const Bil b1 = s.b1;
      const float3 dx1 = s.dx1, dy1 = s.dy1, c1 = s.c1;
      float R1 = (float)E.spec_res[s.l1];
      gs += s.f * R1 * (gsp.x * dx1.x + gsp.y * dx1.y + gsp.z * dx1.z);
      gt += s.f * R1 * (gsp.x * dy1.x + gsp.y * dy1.y + gsp.z * dy1.z);
      eg.b1 = b1;
      eg.w1 = s.f;
      float glod = gsp.x * (c1.x - c0.x) + gsp.y * (c1.y - c0.y) + gsp.z * (c1.z - c0.z);
      grc += glod * (float)(L - 1);
    }
    gwr = cube_coord_grad(cr, gs, gt);
  }
  // irradiance cube at N
  float3 gNh = make_float3(0.f, 0.f, 0.f);
  {
    const CubeCoord& cn = s.cn;
    const Bil bi = s.bi;
    const float3 dx = s.idx, dy = s.idy;
    float3 gi = make_float3(girr3[0], girr3[1], girr3[2]);
    float Ri = (float)E.irr_res;
    float gs = Ri * (gi.x * dx.x + gi.y * dx.y + gi.z * dx.z);
    float gt = Ri * (gi.x * dy.x + gi.y * dy.y + gi.z * dy.z);
    eg.face_n = cn.face;
    eg.bi = bi;
    eg.gir = gi;
    gNh = cube_coord_grad(cn, gs, gt);
  }
  // w_r = 2 nv Nh - wo ; nv = Nh.wo ; ndv = clamp(nv)
  float gnv = 2.f * (s.Nh.x * gwr.x + s.Nh.y * gwr.y + s.Nh.z * gwr.z);
  gNh.x += 2.f * s.nv * gwr.x;
  gNh.y += 2.f * s.nv * gwr.y;
  gNh.z += 2.f * s.nv * gwr.z;
  if (s.nv >= kNdotVMin() && s.nv <= 1.f) gnv += gndv;
  gNh.x += gnv * s.wo.x;
  gNh.y += gnv * s.wo.y;
  gNh.z += gnv * s.wo.z;
  // roughness clamp
  float grough = (s.rough >= 0.f && s.rough <= 1.f) ? grc : 0.f;
  // N -> Nh = N/|N|
  if (s.nz) {
    float inl = 1.f / s.nlen;
    float dp = s.Nh.x * gNh.x + s.Nh.y * gNh.y + s.Nh.z * gNh.z;
    gX[5] = (gNh.x - s.Nh.x * dp) * inl;
    gX[6] = (gNh.y - s.Nh.y * dp) * inl;
    gX[7] = (gNh.z - s.Nh.z * dp) * inl;
  }
  // normalised buffers: lam = X/A etc.
  float iA = 1.f / A;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    gX[c] = glam[c] * iA;
    gA -= glam[c] * s.lam[c] * iA;
  }
  gX[3] = gmet * iA;
  gA -= gmet * s.met * iA;
  gX[4] = grough * iA;
  gA -= grough * s.rough * iA;
}

}  // namespace ts
