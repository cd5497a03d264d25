// Per-fragment evaluation shared by the forward and backward rasterisers.
// Both kernels must take identical decisions (support cut, alpha threshold,
// termination), so the arithmetic lives here once and uses explicit fmaf /
// rounding intrinsics: no contraction choice is left to the compiler.
#pragma once
#include "ts_common.cuh"

namespace ts {

struct Frag {
  float u, v, rd, G, oG, alpha;
};

// Closed-form ray-splat intersection (Sec. 3.1): u = h_u.x / h_w.x,
// v = h_v.x / h_w.x with x = (x', y', 1); Gaussian kernel (Eq. 2); opacity
// alpha = min(0.99, o G).  Returns false when the fragment does not exist
// (outside the 3-sigma support square or alpha < 1/255).
__device__ __forceinline__ bool eval_frag(const Record& r, float xp, float yp, Frag& f) {
  float den = fmaf(r.r1.z, xp, fmaf(r.r1.w, yp, r.r2.x));
  // (un, vn) as one channel pair: same roundings as the scalar fmaf chains
  const float2 uvn = fma2(f2(r.r0.x, r.r0.y), f2(xp, xp), fma2(f2(r.r0.z, r.r0.w), f2(yp, yp), f2(r.r1.x, r.r1.y)));
  f.rd = __fdividef(1.0f, den);
  const float2 uv = mul2(uvn, f2(f.rd, f.rd));
  f.u = uv.x;
  f.v = uv.y;
  if (!(fabsf(f.u) <= 3.0f && fabsf(f.v) <= 3.0f)) return false;
  float q = fmaf(f.u, f.u, __fmul_rn(f.v, f.v));
  f.G = __expf(__fmul_rn(-0.5f, q));
  f.oG = __fmul_rn(r.r2.y, f.G);
  f.alpha = fminf(kAlphaMax(), f.oG);
  return f.alpha >= kAlphaMin();
}

// Conservative test: can splat r make a fragment at any pixel centre of the
// block [x0, x1] x [y0, y1] (centred pixel coordinates)?  The block maps to a
// convex quad in the splat's (u, v) plane with the corner images as vertices
// whenever the homography's denominator keeps its sign over the block; the
// splat is rejected only when all four corners lie beyond the same side of
// the support square |u|, |v| <= 3 by a 0.1 % margin, far above the FP32
// error of any pixel's (u, v), or when the bounding box of the corner images
// lies outside the disc where the opacity cut alpha >= 1/255 can pass.
// Blocks the plane crosses edge-on are kept.
__device__ __forceinline__ bool block_may_hit(const Record& r, float x0, float x1, float y0, float y1) {
  float umin = 3.0e38f, umax = -3.0e38f, vmin = 3.0e38f, vmax = -3.0e38f;
  float dmin = 3.0e38f, dmax = -3.0e38f;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float x = (c & 1) ? x1 : x0, y = (c & 2) ? y1 : y0;
    const float den = fmaf(r.r1.z, x, fmaf(r.r1.w, y, r.r2.x));
    const float2 uvn = fma2(f2(r.r0.x, r.r0.y), f2(x, x), fma2(f2(r.r0.z, r.r0.w), f2(y, y), f2(r.r1.x, r.r1.y)));
    const float rd = __fdividef(1.0f, den);
    const float2 uv = mul2(uvn, f2(rd, rd));
    const float u = uv.x, v = uv.y;
    umin = fminf(umin, u); umax = fmaxf(umax, u);
    vmin = fminf(vmin, v); vmax = fmaxf(vmax, v);
    dmin = fminf(dmin, den); dmax = fmaxf(dmax, den);
  }
  if (!(dmin > 0.f || dmax < 0.f)) return true;
  const float lim = 3.003f;
  if (umin > lim || umax < -lim || vmin > lim || vmax < -lim) return false;
  // alpha >= 1/255 needs o exp(-(u^2 + v^2)/2) >= 1/255, i.e. u^2 + v^2 <=
  // 2 ln(255 o): reject when the box of the corner images misses that disc
  // (0.2 % + 1e-3 margin, far above the FP32 error of (u, v) and of the
  // exponential in eval_frag)
  const float du = fmaxf(fmaxf(umin, -umax), 0.f), dv = fmaxf(fmaxf(vmin, -vmax), 0.f);
  const float r2 = 2.f * __logf(255.f * r.r2.y);
  return fmaf(du, du, dv * dv) <= fmaf(r2, 1.002f, 1e-3f);
}

struct TexSample {
  int ia, ib, ja, jb;
  float fx, fy;
};

// Eq. 5: s = (u + 3)/6, t = (v + 3)/6; texel-centre coordinates x = s T - 1/2.
// A fragment has |u|, |v| <= 3, so x lies in [-1/2, T - 1/2] and floor(x) in
// [-1, T - 1] (the float32 rounding of (u + 3) T/6 stays within the same
// integer parts): clamping the lower corner from below and the upper one
// from above is the whole clamp-to-edge.
__device__ __forceinline__ TexSample tex_setup(float u, float v, int T) {
  TexSample s;
  float Ts6 = (float)T * (1.0f / 6.0f);
  float xs = fmaf(u + 3.0f, Ts6, -0.5f);
  float ys = fmaf(v + 3.0f, Ts6, -0.5f);
  float fi = floorf(xs), fj = floorf(ys);
  s.fx = xs - fi;
  s.fy = ys - fj;
  int i0 = (int)fi, j0 = (int)fj;
  s.ia = max(i0, 0);
  s.ib = min(i0 + 1, T - 1);
  s.ja = max(j0, 0);
  s.jb = min(j0 + 1, T - 1);
  return s;
}

// The four bilinear corners' 8 channels: t0 (ia, ja), t1 (ib, ja), t2 (ia, jb),
// t3 (ib, jb) of the splat's chart.
template <int DT>
__device__ __forceinline__ void tex_corners(const ViewDesc& V, long long splat, int T, const TexSample& s, float t0[8],
                                            float t1[8], float t2[8], float t3[8]) {
  const unsigned ra = (unsigned)(s.ja * T), rb = (unsigned)(s.jb * T);
  if (DT == DT_F32 && V.tex_v8) {
    const float* c = reinterpret_cast<const float*>(V.texels) + splat * (long long)(T * T * 8);
    load_texel_v8(c + (ra + s.ia) * 8u, t0);
    load_texel_v8(c + (ra + s.ib) * 8u, t1);
    load_texel_v8(c + (rb + s.ia) * 8u, t2);
    load_texel_v8(c + (rb + s.ib) * 8u, t3);
  } else {
    const long long base = splat * (long long)T * T;
    load_texel(V.texels, DT, base + ra + s.ia, t0);
    load_texel(V.texels, DT, base + ra + s.ib, t1);
    load_texel(V.texels, DT, base + rb + s.ia, t2);
    load_texel(V.texels, DT, base + rb + s.ib, t3);
  }
}

// Bilinear texel fetch (Eq. 6) of the 8 channels, as 4 channel pairs.
// PHASED (float32 texels in 32-byte loads): the two corners of the upper row
// are loaded and summed before those of the lower row, so 16 texel registers
// are live instead of 32 (the forward instances with indirect light or
// two-component normals, whose other state would otherwise spill, and the
// non-saving ones, where it measured faster); the sums are the same
// operations in the same order either way, so saving and non-saving renders
// give the same image.
template <int DT, bool PHASED = false>
__device__ __forceinline__ void tex_fetch(const ViewDesc& V, long long splat, int T, const TexSample& s,
                                          float out[8]) {
  // the four corner weights (the same products the backward uses)
  const float gx = 1.f - s.fx, gy = 1.f - s.fy;
  const float2 w01 = mul2(f2(gx, s.fx), f2(gy, gy)), w23 = mul2(f2(gx, s.fx), f2(s.fy, s.fy));
  const float2 W0 = f2(w01.x, w01.x), W1 = f2(w01.y, w01.y), W2 = f2(w23.x, w23.x), W3 = f2(w23.y, w23.y);
  if (PHASED && DT == DT_F32 && V.tex_v8) {
    const float* c = reinterpret_cast<const float*>(V.texels) + splat * (long long)(T * T * 8);
    const unsigned ra = (unsigned)(s.ja * T), rb = (unsigned)(s.jb * T);
    float ta[8], tb[8];
    load_texel_v8_ordered(c + (ra + s.ia) * 8u, ta);
    load_texel_v8_ordered(c + (ra + s.ib) * 8u, tb);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = 2 * q;
      const float2 o = fma2(W1, f2(tb[k], tb[k + 1]), mul2(W0, f2(ta[k], ta[k + 1])));
      out[k] = o.x;
      out[k + 1] = o.y;
    }
    load_texel_v8_ordered(c + (rb + s.ia) * 8u, ta);
    load_texel_v8_ordered(c + (rb + s.ib) * 8u, tb);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = 2 * q;
      const float2 o = fma2(W3, f2(tb[k], tb[k + 1]), fma2(W2, f2(ta[k], ta[k + 1]), f2(out[k], out[k + 1])));
      out[k] = o.x;
      out[k + 1] = o.y;
    }
    return;
  }
  float t0[8], t1[8], t2[8], t3[8];
  tex_corners<DT>(V, splat, T, s, t0, t1, t2, t3);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = 2 * q;
    float2 o = mul2(W0, f2(t0[c], t0[c + 1]));
    o = fma2(W1, f2(t1[c], t1[c + 1]), o);
    o = fma2(W2, f2(t2[c], t2[c + 1]), o);
    o = fma2(W3, f2(t3[c], t3[c + 1]), o);
    out[c] = o.x;
    out[c + 1] = o.y;
  }
}

// Hardware-filtered fetch (supplementary Sec. 1): the texel-centre coordinate
// of Eq. 5 inside the splat's chart, clamped to the chart's outer texel
// centres (clamp-to-edge as in the software path, instead of the paper's
// formula, which bleeds half a texel into the neighbouring chart at s, t in
// {0, 1}), offset by the chart origin from the indirection buffer and sampled
// by tex2D with linear filtering from the two 4-channel atlases.  The texture
// unit computes the bilinear weights in fixed point (8 fractional bits).
__device__ __forceinline__ void tex_fetch_hw(const ViewDesc& V, long long splat, int T, float u, float v,
                                             float out[8]) {
  const uint2 ch = V.chart[splat];
  const float Ts6 = (float)T * (1.0f / 6.0f);
  const float hi = (float)(T - 1);
  const float xs = fminf(fmaxf(fmaf(u + 3.0f, Ts6, -0.5f), 0.f), hi);
  const float ys = fminf(fmaxf(fmaf(v + 3.0f, Ts6, -0.5f), 0.f), hi);
  const float x = (float)ch.x + 0.5f + xs, y = (float)ch.y + 0.5f + ys;
  const float4 a = tex2D<float4>(V.atlas2d[0], x, y);
  const float4 b = tex2D<float4>(V.atlas2d[1], x, y);
  out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
  out[4] = b.x; out[5] = b.y; out[6] = b.z; out[7] = b.w;
}

// Two-component tangent normal (Sec. 3.5.1): n_z from the interpolated
// (n_x, n_y), zero outside the unit disc.
__device__ __forceinline__ float rebuild_nz(float nx, float ny) {
  const float r = fmaf(-nx, nx, fmaf(-ny, ny, 1.f));
  return r > 0.f ? sqrtf(r) : 0.f;
}

// Normal mapping (Eq. 7): n = [t_u, t_v, n_f] n^t, in place on x[5..7].
__device__ __forceinline__ void normal_map(const Record& r, float x[8]) {
  float a = x[5], b = x[6], c = x[7];
  const float2 n01 = fma2(f2(a, a), f2(r.r2.z, r.r2.w), fma2(f2(b, b), f2(r.r3.y, r.r3.z), mul2(f2(c, c), f2(r.r4.x, r.r4.y))));
  x[5] = n01.x;
  x[6] = n01.y;
  x[7] = fmaf(a, r.r3.x, fmaf(b, r.r3.w, c * r.r4.z));
}

// ---- indirect light (Eq. 9, Eq. 12): per-splat SH in the reflection direction
// Real SH normalisation constants up to degree 2.
constexpr float kSH0 = 0.28209479177387814f;   // 1 / (2 sqrt(pi))
constexpr float kSH1 = 0.48860251190291992f;   // sqrt(3 / (4 pi))
constexpr float kSH2 = 1.09254843059207907f;   // sqrt(15 / (4 pi))
constexpr float kSH3 = 0.31539156525252005f;   // sqrt(5 / (16 pi))
constexpr float kSH4 = 0.54627421529603959f;   // sqrt(15 / (16 pi))

__device__ __forceinline__ void sh_basis(float3 w, int K, float Y[9]) {
  Y[0] = kSH0;
  if (K > 1) {
    Y[1] = -kSH1 * w.y;
    Y[2] = kSH1 * w.z;
    Y[3] = -kSH1 * w.x;
  }
  if (K > 4) {
    Y[4] = kSH2 * w.x * w.y;
    Y[5] = -kSH2 * w.y * w.z;
    Y[6] = kSH3 * (2.f * w.z * w.z - w.x * w.x - w.y * w.y);
    Y[7] = -kSH2 * w.x * w.z;
    Y[8] = kSH4 * (w.x * w.x - w.y * w.y);
  }
}

// Reflection of w_o about the fragment's normalised normal n_w (w_o when n_w
// vanishes): returns w_r and the pieces the adjoint needs.
struct Refl {
  float3 nh, wr;
  float ndw, inl;
};
__device__ __forceinline__ Refl reflect_dir(float3 nw, float3 wo) {
  Refl r;
  const float n2 = nw.x * nw.x + nw.y * nw.y + nw.z * nw.z;
  if (n2 >= 1e-24f) {
    r.inl = rsqrtf(n2);
    r.nh = make_float3(nw.x * r.inl, nw.y * r.inl, nw.z * r.inl);
  } else {
    r.inl = 0.f;
    r.nh = wo;
  }
  r.ndw = r.nh.x * wo.x + r.nh.y * wo.y + r.nh.z * wo.z;
  r.wr = make_float3(2.f * r.ndw * r.nh.x - wo.x, 2.f * r.ndw * r.nh.y - wo.y, 2.f * r.ndw * r.nh.z - wo.z);
  return r;
}

// l = sum_j c_j Y_j(w_r) for the three channels, and with PROJ also
// s_j = gl . c_j; c rows are [K][3] floats padded to a multiple of 4, read
// as 16-byte vectors (the same address on every lane of the warp).
template <bool PROJ>
__device__ __forceinline__ float3 sh_eval(const float* __restrict__ c, int K, const float Y[9], float3 gl = {},
                                          float s[9] = nullptr) {
  float3 l = make_float3(0.f, 0.f, 0.f);
  if (PROJ) {
#pragma unroll
    for (int j = 0; j < 9; ++j) s[j] = 0.f;
  }
  const float4* c4 = reinterpret_cast<const float4*>(c);
  const int n4 = (3 * K + 3) >> 2;
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    if (q < n4) {
      const float4 a = __ldg(c4 + q);
      const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int e = 4 * q + i, j = e / 3, ch = e - 3 * (e / 3);
        if (e < 27 && j < K) {
          const float x = av[i];
          if (ch == 0) l.x = fmaf(x, Y[j], l.x);
          if (ch == 1) l.y = fmaf(x, Y[j], l.y);
          if (ch == 2) l.z = fmaf(x, Y[j], l.z);
          if (PROJ) s[j] = fmaf(ch == 0 ? gl.x : (ch == 1 ? gl.y : gl.z), x, s[j]);
        }
      }
    }
  }
  return l;
}

// sum_j s_j grad Y_j(w) (the gradient of the basis as written in sh_basis,
// taken on the full space; the reflection adjoint projects it)
__device__ __forceinline__ float3 sh_grad_dir(float3 w, int K, const float s[9]) {
  float3 g = make_float3(0.f, 0.f, 0.f);
  if (K > 1) {
    g.x = -kSH1 * s[3];
    g.y = -kSH1 * s[1];
    g.z = kSH1 * s[2];
  }
  if (K > 4) {
    g.x += kSH2 * (w.y * s[4] - w.z * s[7]) - 2.f * kSH3 * w.x * s[6] + 2.f * kSH4 * w.x * s[8];
    g.y += kSH2 * (w.x * s[4] - w.z * s[5]) - 2.f * kSH3 * w.y * s[6] - 2.f * kSH4 * w.y * s[8];
    g.z += -kSH2 * (w.y * s[5] + w.x * s[7]) + 4.f * kSH3 * w.z * s[6];
  }
  return g;
}

// Rasteriser CTAs: a 16 x 16 tile is 8 pixel blocks of 8 x 4 (one warp
// each), split over kCtasPerTile CTAs of kRasterWarps warps
constexpr int kRasterWarps = 4;
constexpr int kCtasPerTile = 8 / kRasterWarps;

// the tile of this CTA (in launch order) and the 8 x 4 block of this warp;
// a launch order whose sort's bounded wait ran out is not used (the tiles
// are then taken in tile order, which changes no result)
__device__ __forceinline__ int raster_tile(const ViewTable& vt) {
  const int b = (int)blockIdx.x / kCtasPerTile;
  if (!vt.tile_order || (vt.sort_err && __ldcg(vt.sort_err + SORT_FLAG_ORDER))) return b;
  return (int)vt.tile_order[b];
}
// the key lists may be wrong (a bounded wait of the depth sort ran out, or a
// consumer of its order found an id out of range): the forward then writes
// NaN to its pixels and the backward adds nothing
__device__ __forceinline__ bool lists_failed(const ViewTable& vt) {
  return vt.sort_err && __ldcg(vt.sort_err + SORT_FLAG_LISTS);
}
__device__ __forceinline__ int raster_block() {
  return ((int)blockIdx.x % kCtasPerTile) * kRasterWarps + (int)(threadIdx.x >> 5);
}

__device__ __forceinline__ void pixel_of(int tile_local, int tiles_x, int wblk, int& px, int& py) {
  int tx = tile_local % tiles_x, ty = tile_local / tiles_x;
  int lane = threadIdx.x & 31;
  // 8 x 4 pixel block per warp, 2 x 4 blocks per 16 x 16 tile
  px = tx * TILE + (wblk & 1) * 8 + (lane & 7);
  py = ty * TILE + (wblk >> 1) * 4 + (lane >> 3);
}

}  // namespace ts
