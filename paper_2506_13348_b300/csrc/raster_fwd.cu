// Forward rasteriser: one thread per pixel, one warp per 8x4 pixel block;
// a 16x16 tile's 8 blocks are split over two CTAs of 4 warps (the finer
// CTAs refill an SM sooner when their warps finish early), the tiles taken
// longest list first.
//
// Each warp walks the tile's depth-sorted splat list front to back on its
// own (no block-wide barrier), 32 entries at a time:
//   0. lane t's entry has its first 48 bytes (the homography rows and the
//      opacity) copied into shared memory by cp.async one chunk ahead (the
//      copy of chunk k+1 runs while the warp works on chunk k); the lane
//      tests the entry against the warp's whole pixel block (conservative,
//      see block_may_hit): most entries of a tile list miss a given block
//      and are dropped here;
//   1. the warp takes the surviving entries in order: every lane evaluates
//      the entry at its pixel (closed-form (u,v) of the splat, support cut,
//      Gaussian, opacity -- Sec. 3.1, Eq. 2) and the lanes it covers blend
//      it: bilinear texel fetch from the splat's chart (Eq. 5-6), normal
//      mapping (Eq. 7) with the rest of the record, and front-to-back
//      compositing of the 8 G-buffer channels (Eq. 3, 8-9).  All lanes read
//      the same record (a shared-memory broadcast) and mostly the same texels.
// Each pixel blends exactly the fragments of the definition, in order, with
// the same arithmetic.  A warp leaves the list once all its pixels'
// transmittance fell below 1e-4.  Shading (Eq. 10-12) is fused into the
// epilogue; the G-buffer is written only when the backward needs it.
#include "raster.cuh"
#include "shading.cuh"
#include "kernels.h"
#include "prof.h"

namespace ts {

// WIDE: the instance for large grids (kWideTiles tiles or more): 8 CTAs per
// SM at 64 registers instead of 6 at 80, the texel corners loaded in two
// phases to fit; it pays once the grid is many waves deep (4 views of 800x800:
// 2.021 -> 1.968 ms) and loses on a single view's grid (0.614 -> 0.674 ms),
// where the longer per-CTA time stretches the last wave.  Same arithmetic,
// same image.
template <int DT, bool SAVE, bool STATS, int SMP, int FEAT = 0, bool WIDE = false>
__global__ void __launch_bounds__(32 * kRasterWarps, WIDE ? 8 : 3 * kCtasPerTile) k_raster_fwd(ViewTable vt, const Record* __restrict__ rec,
                                                     const uint32_t* __restrict__ pair_items,
                                                     const uint2* __restrict__ ranges, FragCounters stats) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr bool IND = (FEAT & FEAT_IND) != 0, N2 = (FEAT & FEAT_N2) != 0;
  const int tile = raster_tile(vt);
  if ((unsigned)tile >= (unsigned)vt.n_tiles) return;  // an order from a failed sort (flag set)
  const int v = find_view(vt, tile);
  const ViewDesc& V = vt.v[v];
  int px, py;
  pixel_of(tile - V.tile_off, V.tiles_x, raster_block(), px, py);
  const bool inside = px < V.W && py < V.H;
  if (lists_failed(vt)) {  // reported by the host; the image is marked invalid
    if (inside) V.rgba[py * V.W + px] = make_float4(__int_as_float(0x7fffffff), __int_as_float(0x7fffffff),
                                                    __int_as_float(0x7fffffff), __int_as_float(0x7fffffff));
    return;
  }
  const float xp = (float)px + 0.5f - V.cx;
  const float yp = (float)py + 0.5f - V.cy;
  const uint2 range = ranges[tile];
  const int T = V.T;
  const int lane = threadIdx.x & 31;
  // the warp's 8x4 pixel block in centred pixel coordinates (for culling)
  const float bx0 = (float)(px - (lane & 7)) + 0.5f - V.cx, bx1 = bx0 + 7.f;
  const float by0 = (float)(py - (lane >> 3)) + 0.5f - V.cy, by1 = by0 + 3.f;

  float Tr = 1.f;
  float Acc = 0.f;  // coverage as the blended sum (Eq. 3 with a = 1): exact where 1 - T cancels
  float Zs = 0.f;   // blended camera depth of the hits (saved renders)
  float X[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) X[c] = 0.f;
  int last = -1;
  int stop = -1;  // list index at which the pixel terminated (statistics)
  bool done = !inside;
  unsigned n_blend = 0;
  // indirect light: w_o of the pixel and the blended SH light of the fragments
  float3 wo = make_float3(0.f, 0.f, 1.f);
  float Xi[3] = {0.f, 0.f, 0.f};
  const int shK = (V.sh_deg + 1) * (V.sh_deg + 1);
  if (IND) {
    const float3 d = world_ray(V, xp, yp);
    const float id = rsqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
    wo = make_float3(-d.x * id, -d.y * id, -d.z * id);
  }

  // per-warp walk: no CTA barrier; lane t stages entry c0 + t's first 48
  // bytes in shared memory for the block test and the lockstep loop.  The
  // records of the next chunk are copied asynchronously (cp.async) while
  // the warp works on the current one; the item ids run one chunk further
  // ahead in a register.
  {
    __shared__ __align__(16) float4 s_r[kRasterWarps][2][32][3];
    __shared__ uint32_t s_it[kRasterWarps][2][32];
    const int warp = threadIdx.x >> 5;
    auto issue = [&](int b, unsigned c, uint32_t it) {
      if (c + lane < range.y) {
        const float4* rp = reinterpret_cast<const float4*>(rec + it);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const unsigned dst = (unsigned)__cvta_generic_to_shared(&s_r[warp][b][lane][q]);
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(rp + q) : "memory");
        }
        s_it[warp][b][lane] = it;
      }
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    uint32_t it_next = (range.x + lane < range.y) ? __ldg(pair_items + range.x + lane) : 0u;
    issue(0, range.x, it_next);
    it_next = (range.x + 32 + lane < range.y) ? __ldg(pair_items + range.x + 32 + lane) : 0u;
    int b = 0;
    for (unsigned c0 = range.x; c0 < range.y; c0 += 32, b ^= 1) {
      if (__all_sync(FULL, done)) break;
      issue(b ^ 1, c0 + 32, it_next);  // next chunk's records
      it_next = (c0 + 64 + lane < range.y) ? __ldg(pair_items + c0 + 64 + lane) : 0u;
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // this chunk's records are in
      __syncwarp();
      const unsigned e = c0 + lane;
      bool cand = false;
      if (e < range.y) {
        Record c;
        c.r0 = s_r[warp][b][lane][0];
        c.r1 = s_r[warp][b][lane][1];
        c.r2 = s_r[warp][b][lane][2];
        cand = block_may_hit(c, bx0, bx1, by0, by1);
      }
      const unsigned cmask = __ballot_sync(FULL, cand);
      for (unsigned m = cmask; m; m &= m - 1) {
        const int t = __ffs(m) - 1;
        Record r;
        r.r0 = s_r[warp][b][t][0];
        r.r1 = s_r[warp][b][t][1];
        r.r2 = s_r[warp][b][t][2];
        Frag f;
        const bool ok = !done && eval_frag(r, xp, yp, f);
        if (__any_sync(FULL, ok)) {
          const float4* rp = reinterpret_cast<const float4*>(rec + s_it[warp][b][t]);
          r.r3 = __ldg(rp + 3);
          r.r4 = __ldg(rp + 4);
          if (ok) {
            const long long splat = (long long)s_it[warp][b][t] - V.item_off;
            float x[8];
            if (SMP == SMP_SOFTWARE) {
              const TexSample ts_ = tex_setup(f.u, f.v, T);
              tex_fetch<DT, FEAT != 0 || !SAVE || WIDE>(V, splat, T, ts_, x);
              if (STATS) {  // the four texels this fragment reads
                uint32_t* w = stats.touched + (size_t)s_it[warp][b][t] * stats.words_per_item;
                const int q0 = ts_.ja * T + ts_.ia, q1 = ts_.ja * T + ts_.ib;
                const int q2 = ts_.jb * T + ts_.ia, q3 = ts_.jb * T + ts_.ib;
                atomicOr(w + (q0 >> 5), 1u << (q0 & 31));
                atomicOr(w + (q1 >> 5), 1u << (q1 & 31));
                atomicOr(w + (q2 >> 5), 1u << (q2 & 31));
                atomicOr(w + (q3 >> 5), 1u << (q3 & 31));
              }
            } else if (SMP == SMP_HW_ATLAS) {
              tex_fetch_hw(V, splat, T, f.u, f.v, x);
            } else {
              load_texel(V.texels, DT, splat * (long long)T * T, x);
            }
            if (N2) x[7] = rebuild_nz(x[5], x[6]);
            normal_map(r, x);
            const float w = f.alpha * Tr;
            if (IND && V.sh) {
              // the splat's SH light in the reflection direction of this
              // fragment's normal (Eq. 9: blended like the other channels)
              const Refl rf = reflect_dir(make_float3(x[5], x[6], x[7]), wo);
              float Y[9];
              sh_basis(rf.wr, shK, Y);
              const float3 l = sh_eval<false>(V.sh + splat * V.sh_stride, shK, Y);
              Xi[0] = fmaf(w, l.x, Xi[0]);
              Xi[1] = fmaf(w, l.y, Xi[1]);
              Xi[2] = fmaf(w, l.z, Xi[2]);
            }
            const float2 W2 = f2(w, w);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float2 o = fma2(W2, f2(x[2 * q], x[2 * q + 1]), f2(X[2 * q], X[2 * q + 1]));
              X[2 * q] = o.x;
              X[2 * q + 1] = o.y;
            }
            Acc += w;
            if (SAVE) Zs = fmaf(w, r.r4.w * f.rd, Zs);  // depth channel: z = D / den
            Tr = Tr * (1.f - f.alpha);
            last = (int)(c0 + t);
            if (STATS) ++n_blend;
            if (Tr < kTMin()) {
              done = true;
              stop = last;
            }
          }
        }
      }
      __syncwarp();
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
  }

  if (inside) {
    const int pix = py * V.W + px;
    const float A = Acc;
    float3 d = world_ray(V, xp, yp);
    V.rgba[pix] = IND ? shade_pixel(V.env, X, A, d, nullptr, Xi, V.vis ? V.vis[pix] : 1.f)
                      : shade_pixel(V.env, X, A, d, nullptr);
    if (SAVE && IND) V.gind[pix] = make_float4(Xi[0], Xi[1], Xi[2], 0.f);
    if (SAVE) {
      V.gbuf[2 * pix] = make_float4(X[0], X[1], X[2], X[3]);
      V.gbuf[2 * pix + 1] = make_float4(X[4], X[5], X[6], X[7]);
      V.trans[pix] = Tr;
      V.acc[pix] = Acc;
      V.zsum[pix] = Zs;
      V.last[pix] = last;
    }
  }
  if (STATS) {
    // evaluated fragments of the definition: list entries up to and including
    // the one that terminated the pixel (the whole list if it never did)
    unsigned long long e = inside ? (unsigned long long)((stop >= 0 ? stop + 1 : (int)range.y) - (int)range.x) : 0ull;
    unsigned long long b = n_blend;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(FULL, e, o);
      b += __shfl_xor_sync(FULL, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(stats.counts + 0, e);
      atomicAdd(stats.counts + 1, b);
    }
  }
}

namespace {

// grids of at least this many tiles take the WIDE instance of the saving
// forward (4 views of 800x800: 10 000 tiles; one view: 2 500)
constexpr int kWideTiles = 8192;

template <int DT, bool SAVE, bool STATS, int SMP>
void launch_feat(int feat, dim3 grid, dim3 block, cudaStream_t st, const ViewTable& vt, const Record* rec,
                 const uint32_t* pair_items, const uint2* ranges, FragCounters stats) {
  switch (feat & (FEAT_IND | FEAT_N2)) {
    case 0:
      if constexpr (SAVE && !STATS && SMP == SMP_SOFTWARE) {
        if (vt.n_tiles >= kWideTiles) {
          k_raster_fwd<DT, SAVE, STATS, SMP, 0, true><<<grid, block, 0, st>>>(vt, rec, pair_items, ranges, stats);
          break;
        }
      }
      k_raster_fwd<DT, SAVE, STATS, SMP, 0><<<grid, block, 0, st>>>(vt, rec, pair_items, ranges, stats);
      break;
    case FEAT_N2:
      k_raster_fwd<DT, SAVE, STATS, SMP, FEAT_N2><<<grid, block, 0, st>>>(vt, rec, pair_items, ranges, stats);
      break;
    case FEAT_IND:
      k_raster_fwd<DT, SAVE, STATS, SMP, FEAT_IND><<<grid, block, 0, st>>>(vt, rec, pair_items, ranges, stats);
      break;
    default:
      k_raster_fwd<DT, SAVE, STATS, SMP, FEAT_IND | FEAT_N2><<<grid, block, 0, st>>>(vt, rec, pair_items, ranges,
                                                                                       stats);
  }
}

// samplers without indirect light (the host rejects that combination)
template <int DT, int SMP>
void launch_feat_n2(int feat, dim3 grid, dim3 block, cudaStream_t st, const ViewTable& vt, const Record* rec,
                    const uint32_t* pair_items, const uint2* ranges) {
  if (feat & FEAT_N2)
    k_raster_fwd<DT, false, false, SMP, FEAT_N2><<<grid, block, 0, st>>>(vt, rec, pair_items, ranges, FragCounters{});
  else
    k_raster_fwd<DT, false, false, SMP, 0><<<grid, block, 0, st>>>(vt, rec, pair_items, ranges, FragCounters{});
}

template <int DT>
void launch_dt(const ViewTable& vt, const Record* rec, const uint32_t* pair_items, const uint2* ranges, bool save,
               const FragCounters* stats, int sampler, int feat, cudaStream_t st) {
  dim3 grid(vt.n_tiles * kCtasPerTile), block(32 * kRasterWarps);
  if (sampler == SMP_FLAT)
    launch_feat_n2<DT, SMP_FLAT>(feat, grid, block, st, vt, rec, pair_items, ranges);
  else if (stats)  // fragment statistics: the features change no fragment
    k_raster_fwd<DT, false, true, SMP_SOFTWARE><<<grid, block, 0, st>>>(vt, rec, pair_items, ranges, *stats);
  else if (save)
    launch_feat<DT, true, false, SMP_SOFTWARE>(feat, grid, block, st, vt, rec, pair_items, ranges, FragCounters{});
  else
    launch_feat<DT, false, false, SMP_SOFTWARE>(feat, grid, block, st, vt, rec, pair_items, ranges, FragCounters{});
}

}  // namespace

void launch_raster_fwd(const ViewTable& vt, const Record* rec, const uint32_t* pair_items,
                       const uint2* ranges, int tex_dtype, bool save, const FragCounters* stats, int sampler,
                       int feat, cudaStream_t st) {
  if (sampler == SMP_HW_ATLAS) {  // inference only; the atlas dtype is the texture's
    launch_feat_n2<DT_F32, SMP_HW_ATLAS>(feat, dim3(vt.n_tiles * kCtasPerTile), dim3(32 * kRasterWarps), st, vt, rec, pair_items, ranges);
  } else if (tex_dtype == DT_F32) {
    launch_dt<DT_F32>(vt, rec, pair_items, ranges, save, stats, sampler, feat, st);
  } else if (tex_dtype == DT_BF16) {
    launch_dt<DT_BF16>(vt, rec, pair_items, ranges, save, stats, sampler, feat, st);
  } else {
    launch_dt<DT_F16>(vt, rec, pair_items, ranges, save, stats, sampler, feat, st);
  }
  note_launches(1);
}

// Packs the stored charts ([n][T][T][8], any dtype) into the two 4-channel
// 2-D atlases: chart k at texel origin ((k mod charts_x) T, (k div charts_x) T),
// rows indexing t (v) and columns s (u), and records the origin per splat.
__global__ void k_pack_atlas2d(const void* __restrict__ texels, int dtype, long long n, int T, int charts_x,
                               cudaSurfaceObject_t s0, cudaSurfaceObject_t s1, uint2* __restrict__ chart,
                               const uint32_t* __restrict__ chart_of, int half_store) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long tt = (long long)T * T;
  if (i >= n * tt) return;
  const long long k = i / tt;
  const int r = (int)(i - k * tt), jj = r / T, ii = r - jj * T;
  float v[8];
  load_texel(texels, dtype, i, v);
  const long long slot = chart_of ? (long long)chart_of[k] : k;  // chart position of splat k
  const int cx = (int)(slot % charts_x) * T, cy = (int)(slot / charts_x) * T;
  const int x = cx + ii, y = cy + jj;
  if (half_store) {
    const ushort4 a = make_ushort4(__half_as_ushort(__float2half_rn(v[0])), __half_as_ushort(__float2half_rn(v[1])),
                                   __half_as_ushort(__float2half_rn(v[2])), __half_as_ushort(__float2half_rn(v[3])));
    const ushort4 b = make_ushort4(__half_as_ushort(__float2half_rn(v[4])), __half_as_ushort(__float2half_rn(v[5])),
                                   __half_as_ushort(__float2half_rn(v[6])), __half_as_ushort(__float2half_rn(v[7])));
    surf2Dwrite(a, s0, x * (int)sizeof(ushort4), y);
    surf2Dwrite(b, s1, x * (int)sizeof(ushort4), y);
  } else {
    surf2Dwrite(make_float4(v[0], v[1], v[2], v[3]), s0, x * (int)sizeof(float4), y);
    surf2Dwrite(make_float4(v[4], v[5], v[6], v[7]), s1, x * (int)sizeof(float4), y);
  }
  if (r == 0) chart[k] = make_uint2((unsigned)cx, (unsigned)cy);
}

void launch_pack_atlas2d(const void* texels, int dtype, long long n, int T, int charts_x, cudaSurfaceObject_t s0,
                         cudaSurfaceObject_t s1, uint2* chart, const uint32_t* chart_of, int half_store,
                         cudaStream_t st) {
  const long long total = n * (long long)T * T;
  if (total <= 0) return;
  k_pack_atlas2d<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(texels, dtype, n, T, charts_x, s0, s1, chart,
                                                                   chart_of, half_store);
  note_launches(1);
}

// ---- locality-aware chart order: Morton codes of the splat centres ----------
// Order-preserving float <-> uint32 map for atomic min / max of floats.
__device__ __forceinline__ uint32_t f2ord(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// bbox[0..2] = min, bbox[3..5] = max of the centres, as ordered uints
// (initialised to max / min by the caller).
__global__ void k_centre_bbox(const float4* __restrict__ means, long long n, uint32_t* __restrict__ bbox) {
  uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float4 p = means[i];
    const float v[3] = {p.x, p.y, p.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lo[a] = min(lo[a], f2ord(v[a]));
      hi[a] = max(hi[a], f2ord(v[a]));
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = __reduce_min_sync(0xffffffffu, lo[a]);
    hi[a] = __reduce_max_sync(0xffffffffu, hi[a]);
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      atomicMin(bbox + a, lo[a]);
      atomicMax(bbox + 3 + a, hi[a]);
    }
  }
}

__device__ __forceinline__ uint32_t spread3(uint32_t v) {  // 10 bits -> every third bit
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// 30-bit Morton code of each centre in its bounding box, and the splat id.
__global__ void k_morton(const float4* __restrict__ means, long long n, const uint32_t* __restrict__ bbox,
                         uint32_t* __restrict__ codes, uint32_t* __restrict__ ids) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 p = means[i];
  const float v[3] = {p.x, p.y, p.z};
  uint32_t q[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float lo = ord2f(bbox[a]), hi = ord2f(bbox[3 + a]);
    const float t = hi > lo ? (v[a] - lo) / (hi - lo) : 0.f;
    q[a] = (uint32_t)fminf(fmaxf(t * 1024.f, 0.f), 1023.f);
  }
  codes[i] = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
  ids[i] = (uint32_t)i;
}

__global__ void k_chart_of(const uint32_t* __restrict__ ids_sorted, long long n, uint32_t* __restrict__ chart_of) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) chart_of[ids_sorted[r]] = (uint32_t)r;
}

void launch_morton_order(const float4* means, long long n, uint32_t* bbox, uint32_t* codes, uint32_t* ids,
                         cudaStream_t st) {
  if (n <= 0) return;
  const uint32_t init[6] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u};
  cudaMemcpyAsync(bbox, init, sizeof(init), cudaMemcpyHostToDevice, st);
  k_centre_bbox<<<148 * 4, 256, 0, st>>>(means, n, bbox);
  k_morton<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(means, n, bbox, codes, ids);
  note_launches(2);
}

void launch_chart_of(const uint32_t* ids_sorted, long long n, uint32_t* chart_of, cudaStream_t st) {
  if (n <= 0) return;
  k_chart_of<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ids_sorted, n, chart_of);
  note_launches(1);
}

}  // namespace ts
