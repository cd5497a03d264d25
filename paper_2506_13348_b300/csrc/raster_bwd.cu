// Backward rasteriser: one CTA per 16x16 tile, one thread per pixel.
//
// Prologue: the shading adjoint (Eq. 10-12) turns dL/drgba into dL/dX (the
// 8 G-buffer channels) and dL/dA, scattering environment gradients.
// Main loop: the tile's list is walked back to front from the last
// fragment any pixel of the tile blended, recomputing each fragment's (u,v),
// alpha and texel value from the record (the per-pixel fragment lists are
// never stored), recovering the transmittance in front of it by division
// (alpha <= 0.99) and the colour behind it by the usual recurrence.  The
// gradients of a fragment w.r.t. its splat's record (19 values) are summed
// over the warp with a butterfly reduce-scatter (31 shuffles for 32 values)
// and added once per warp; texel gradients go out as 16-byte vector
// reductions.
#include "raster.cuh"
#include "shading.cuh"
#include "kernels.h"
#include "prof.h"

namespace ts {

// Butterfly reduce-scatter: on return lane L holds the warp sum of v[L].
__device__ __forceinline__ float warp_reduce_scatter32(float v[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int step = 16, cnt = 16; step >= 1; step >>= 1, cnt >>= 1) {
    const bool upper = lane & step;
#pragma unroll
    for (int k = 0; k < cnt; ++k) {
      const float send = upper ? v[k] : v[k + cnt];
      const float keep = upper ? v[k + cnt] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, step);
    }
  }
  return v[0];
}

template <int DT>
__global__ void __launch_bounds__(256) k_raster_bwd(ViewTable vt, const Record* __restrict__ rec,
                                                     const uint32_t* __restrict__ pair_items,
                                                     const uint2* __restrict__ ranges, float* __restrict__ g_items,
                                                     GradTable g) {
  __shared__ Record srec[256];
  __shared__ uint32_t sitem[256];
  __shared__ int s_hi;
  const int tile = blockIdx.x;
  const int v = find_view(vt, tile);
  const ViewDesc& V = vt.v[v];
  int px, py;
  pixel_of(tile - V.tile_off, V.tiles_x, px, py);
  const bool inside = px < V.W && py < V.H;
  const float xp = (float)px + 0.5f - V.cx;
  const float yp = (float)py + 0.5f - V.cy;
  const uint2 range = ranges[tile];
  const int T = V.T;
  const float Ts6 = (float)T * (1.0f / 6.0f);

  float gX[8], gA = 0.f, Tcur = 1.f;
  int last = -1;
#pragma unroll
  for (int c = 0; c < 8; ++c) gX[c] = 0.f;
  if (threadIdx.x == 0) s_hi = -1;
  if (inside) {
    const int pix = py * V.W + px;
    const float4 a = V.gbuf[2 * pix], b = V.gbuf[2 * pix + 1];
    const float X[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    Tcur = V.trans[pix];
    last = V.last[pix];
    const float4 dl = V.dl[pix];
    shade_pixel_bwd(V.env, X, 1.f - Tcur, world_ray(V, xp, yp), dl, gX, gA, g.spec, g.irr);
  }
  __syncthreads();
  if (last >= 0) atomicMax(&s_hi, last);
  __syncthreads();
  const int hi_all = s_hi;

  float S[8], SA = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) S[c] = 0.f;
  const int lane = threadIdx.x & 31;

  for (int hi = hi_all; hi >= (int)range.x; hi -= 256) {
    const int lo = max((int)range.x, hi - 255);
    __syncthreads();
    {
      const int i = lo + (int)threadIdx.x;
      if (i <= hi) {
        const uint32_t it = pair_items[i];
        sitem[threadIdx.x] = it;
        srec[threadIdx.x] = rec[it];
      }
    }
    __syncthreads();
    for (int j = hi; j >= lo; --j) {
      const Record r = srec[j - lo];
      float gi[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) gi[k] = 0.f;
      Frag f;
      const bool ok = (j <= last) && eval_frag(r, xp, yp, f);
      if (ok) {
        const TexSample ts_ = tex_setup(f.u, f.v, T);
        const long long splat = (long long)__float_as_int(r.r4.w);
        float x[8], cr[4][8];
        tex_fetch<DT>(V.texels, splat, T, ts_, x, cr);
        const float nt0 = x[5], nt1 = x[6], nt2 = x[7];
        normal_map(r, x);
        const float om = 1.f - f.alpha;
        const float Tb = Tcur / om;
        float ga = 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) ga += gX[c] * (x[c] - S[c]);
        ga += gA * (1.f - SA);
        ga *= Tb;
#pragma unroll
        for (int c = 0; c < 8; ++c) S[c] = f.alpha * x[c] + om * S[c];
        SA = f.alpha + om * SA;
        const float wgt = f.alpha * Tb;
        Tcur = Tb;
        float gx[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) gx[c] = wgt * gX[c];
        // alpha = min(0.99, o G)
        float go = 0.f, gG = 0.f;
        if (f.oG <= kAlphaMax()) {
          go = ga * f.G;
          gG = ga * r.r2.y;
        }
        float gu = -gG * f.G * f.u, gv = -gG * f.G * f.v;
        // normal mapping adjoint: x[5..7] = nt0 t_u + nt1 t_v + nt2 n_f
        const float gn0 = gx[5], gn1 = gx[6], gn2 = gx[7];
        float t8[8];
        t8[0] = gx[0]; t8[1] = gx[1]; t8[2] = gx[2]; t8[3] = gx[3]; t8[4] = gx[4];
        t8[5] = r.r2.z * gn0 + r.r2.w * gn1 + r.r3.x * gn2;
        t8[6] = r.r3.y * gn0 + r.r3.z * gn1 + r.r3.w * gn2;
        t8[7] = r.r4.x * gn0 + r.r4.y * gn1 + r.r4.z * gn2;
        gi[10] = nt0 * gn0; gi[11] = nt0 * gn1; gi[12] = nt0 * gn2;
        gi[13] = nt1 * gn0; gi[14] = nt1 * gn1; gi[15] = nt1 * gn2;
        gi[16] = nt2 * gn0; gi[17] = nt2 * gn1; gi[18] = nt2 * gn2;
        // bilinear adjoint: texel gradients and d/du, d/dv
        const float fx = ts_.fx, fy = ts_.fy, hx = 1.f - fx, hy = 1.f - fy;
        float dxs = 0.f, dys = 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          dxs += t8[c] * (hy * (cr[1][c] - cr[0][c]) + fy * (cr[3][c] - cr[2][c]));
          dys += t8[c] * (hx * (cr[2][c] - cr[0][c]) + fx * (cr[3][c] - cr[1][c]));
        }
        gu += dxs * Ts6;
        gv += dys * Ts6;
        if (g.texels) {
          const long long base = splat * (long long)T * T;
          const long long idx[4] = {base + ts_.ja * T + ts_.ia, base + ts_.ja * T + ts_.ib,
                                    base + ts_.jb * T + ts_.ia, base + ts_.jb * T + ts_.ib};
          const float w4[4] = {hx * hy, fx * hy, hx * fy, fx * fy};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (w4[k] != 0.f) {
              float* p = g.texels + idx[k] * 8;
              red_add_v4(p, w4[k] * t8[0], w4[k] * t8[1], w4[k] * t8[2], w4[k] * t8[3]);
              red_add_v4(p + 4, w4[k] * t8[4], w4[k] * t8[5], w4[k] * t8[6], w4[k] * t8[7]);
            }
          }
        }
        // u = un / den, v = vn / den
        const float gun = gu * f.rd, gvn = gv * f.rd;
        const float gden = -(gu * f.u + gv * f.v) * f.rd;
        gi[0] = gun * xp; gi[1] = gun * yp; gi[2] = gun;
        gi[3] = gvn * xp; gi[4] = gvn * yp; gi[5] = gvn;
        gi[6] = gden * xp; gi[7] = gden * yp; gi[8] = gden;
        gi[9] = go;
      }
      if (__any_sync(0xffffffffu, ok)) {
        const float tot = warp_reduce_scatter32(gi);
        if (lane < 19 && tot != 0.f) red_add(g_items + (size_t)sitem[j - lo] * 20 + lane, tot);
      }
    }
  }
}

void launch_raster_bwd(const ViewTable& vt, const Record* rec, const uint32_t* pair_items,
                       const uint2* ranges, int tex_dtype, float* g_items, const GradTable& g,
                       cudaStream_t st) {
  dim3 grid(vt.n_tiles), block(256);
  if (tex_dtype == DT_F32)
    k_raster_bwd<DT_F32><<<grid, block, 0, st>>>(vt, rec, pair_items, ranges, g_items, g);
  else if (tex_dtype == DT_BF16)
    k_raster_bwd<DT_BF16><<<grid, block, 0, st>>>(vt, rec, pair_items, ranges, g_items, g);
  else
    k_raster_bwd<DT_F16><<<grid, block, 0, st>>>(vt, rec, pair_items, ranges, g_items, g);
  note_launches(1);
}

}  // namespace ts
