// Forward rasteriser: one CTA per 16x16 tile, one thread per pixel.
//
// The tile's depth-sorted splat list is walked front to back in batches of
// 256 records staged in shared memory (one coalesced 80-byte record load
// per thread).  Each pixel evaluates the closed-form (u, v) of every listed
// splat, the Gaussian and the opacity, fetches the bilinear texel of the
// splat's chart, maps the tangent normal to world space and blends the 8
// G-buffer channels (Eq. 3, Eq. 8-9).  The CTA leaves the list as soon as
// every pixel's transmittance fell below 1e-4 (block-wide vote).  Shading
// (Eq. 10-12) is fused into the epilogue, so the G-buffer is written only
// when the caller keeps it for the backward.
#include "raster.cuh"
#include "shading.cuh"
#include "kernels.h"
#include "prof.h"

namespace ts {

template <int DT, bool SAVE, bool STATS>
__global__ void __launch_bounds__(256) k_raster_fwd(ViewTable vt, const Record* __restrict__ rec,
                                                     const uint32_t* __restrict__ pair_items,
                                                     const uint2* __restrict__ ranges,
                                                     unsigned long long* __restrict__ stats) {
  __shared__ Record srec[256];
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

  float Tr = 1.f;
  float X[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) X[c] = 0.f;
  int last = -1;
  bool done = !inside;
  unsigned n_eval = 0, n_blend = 0;

  for (unsigned base = range.x; base < range.y; base += 256) {
    if (__syncthreads_count(done) == 256) break;
    const unsigned i = base + threadIdx.x;
    if (i < range.y) srec[threadIdx.x] = rec[pair_items[i]];
    __syncthreads();
    const int nb = min(256u, range.y - base);
    for (int j = 0; j < nb && !done; ++j) {
      const Record r = srec[j];
      if (STATS) ++n_eval;
      Frag f;
      if (!eval_frag(r, xp, yp, f)) continue;
      TexSample ts_ = tex_setup(f.u, f.v, T);
      float x[8];
      tex_fetch<DT>(V.texels, (long long)__float_as_int(r.r4.w), T, ts_, x, nullptr);
      normal_map(r, x);
      const float w = f.alpha * Tr;
#pragma unroll
      for (int c = 0; c < 8; ++c) X[c] = fmaf(w, x[c], X[c]);
      Tr = Tr * (1.f - f.alpha);
      last = (int)(base + j);
      if (STATS) ++n_blend;
      if (Tr < kTMin()) done = true;
    }
  }

  if (inside) {
    const int pix = py * V.W + px;
    const float A = 1.f - Tr;
    float3 d = world_ray(V, xp, yp);
    V.rgba[pix] = shade_pixel(V.env, X, A, d, nullptr);
    if (SAVE) {
      V.gbuf[2 * pix] = make_float4(X[0], X[1], X[2], X[3]);
      V.gbuf[2 * pix + 1] = make_float4(X[4], X[5], X[6], X[7]);
      V.trans[pix] = Tr;
      V.last[pix] = last;
    }
  }
  if (STATS) {
    unsigned long long e = n_eval, b = n_blend;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(stats + 0, e);
      atomicAdd(stats + 1, b);
    }
  }
}

void launch_raster_fwd(const ViewTable& vt, const Record* rec, const uint32_t* pair_items,
                       const uint2* ranges, int tex_dtype, bool save, unsigned long long* stats,
                       cudaStream_t st) {
  dim3 grid(vt.n_tiles), block(256);
#define TS_LAUNCH(DTV)                                                                         \
  if (stats)                                                                                   \
    k_raster_fwd<DTV, false, true><<<grid, block, 0, st>>>(vt, rec, pair_items, ranges, stats); \
  else if (save)                                                                               \
    k_raster_fwd<DTV, true, false><<<grid, block, 0, st>>>(vt, rec, pair_items, ranges, stats); \
  else                                                                                         \
    k_raster_fwd<DTV, false, false><<<grid, block, 0, st>>>(vt, rec, pair_items, ranges, stats);
  if (tex_dtype == DT_F32) {
    TS_LAUNCH(DT_F32)
  } else if (tex_dtype == DT_BF16) {
    TS_LAUNCH(DT_BF16)
  } else {
    TS_LAUNCH(DT_F16)
  }
#undef TS_LAUNCH
  note_launches(1);
}

}  // namespace ts
