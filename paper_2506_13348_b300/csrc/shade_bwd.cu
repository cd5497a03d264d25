// Shading adjoint (Eq. 10-12) as its own pass over all pixels of a batch.
//
// Each pixel turns dL/drgba into dL/dX (8 G-buffer channels) and dL/dA,
// adds the depth-normal loss's dL/dN, dL/dA and dL/d(blended depth) when
// the view has them, writes them for the backward rasteriser (3 x float4 per
// pixel: X 0-3, X 4-7, (A, depth)), and scatters
// its gradient into the environment maps with bilinear / trilinear weights.
// Environment maps are small and every pixel of a view hits them, so
// atomics on them contend heavily: lanes that hit the same bilinear cell
// are summed over the warp first (warp_cell_scatter), and when all levels and
// the irradiance cube fit (<= 96 KB of float32 gradients) each CTA
// accumulates them in shared memory and adds its copy to the global gradient
// once at the end (persistent grid, a few CTAs per SM).
#include <atomic>

#include "kernels.h"
#include "prof.h"
#include "shading.cuh"

namespace ts {

constexpr int SB_THREADS = 512;
constexpr int SB_MAX_SMEM_FLOATS = 24 * 1024;  // 96 KB

// Offsets of each level / the irradiance cube inside one flat gradient array.
struct EnvGradLayout {
  int off[MAX_LEVELS];
  int irr_off;
  int total;
};

// Where environment gradients go: the CTA's shared-memory copy (flat, levels
// then irradiance) or the global per-level arrays.
struct EnvTarget {
  float* smem;            // non-null: shared copy, offsets lay.off / lay.irr_off
  const GradTable* g;     // else global
  const EnvGradLayout* lay;
  int levels;
  __device__ float* base(int level) const {
    if (smem) return smem + (level < levels ? lay->off[level] : lay->irr_off);
    return level < levels ? g->spec[level] : g->irr;
  }
};

// Adds g (3 channels) x bilinear weights x scale of every live lane into the
// four texels of its cell at `level` (levels = the irradiance cube).
// Neighbouring pixels mostly fall in the same cell of these small maps, so
// per-lane atomics would serialise on a few addresses: lanes are grouped by
// (level, cell); a lane whose cell at most two live lanes share adds its own
// values, each larger group is summed over the warp by a reduce-scatter (12
// values in 16 slots, 13 shuffles) and 12 lanes add the group's totals.
// Every lane of the warp must call this (warp-uniform control flow).
__device__ __forceinline__ void warp_cell_scatter(const EnvTarget& tg, bool live, int level, int R, int face,
                                                  const Bil& b, float3 g, float scale) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned t0 = (unsigned)(face * R * R + b.ja * R + b.ia);
  const unsigned dx = b.ib != b.ia, dy = b.jb != b.ja;
  const unsigned key = live ? (((unsigned)level << 27) | (t0 << 2) | (dx << 1) | dy) : FULL;
  const float hx = 1.f - b.fx, hy = 1.f - b.fy;
  const float w[4] = {hx * hy * scale, b.fx * hy * scale, hx * b.fy * scale, b.fx * b.fy * scale};
  const unsigned livem = __ballot_sync(FULL, live);
  const unsigned same = __match_any_sync(FULL, key) & livem;
  const bool direct = live && __popc(same) <= 2;
  if (direct) {
    float* base = tg.base(level);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (w[k] == 0.f) continue;
      float* p = base + 3 * (t0 + ((k & 1) ? dx : 0u) + ((k & 2) ? dy * (unsigned)R : 0u));
      if (tg.smem) {
        atomicAdd(p, w[k] * g.x);
        atomicAdd(p + 1, w[k] * g.y);
        atomicAdd(p + 2, w[k] * g.z);
      } else {
        red_add(p, w[k] * g.x);
        red_add(p + 1, w[k] * g.y);
        red_add(p + 2, w[k] * g.z);
      }
    }
  }
  const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4, u2 = lane & 2;
  unsigned pend = __ballot_sync(FULL, live && !direct);
  while (pend) {  // warp-uniform
    const int ldr = __ffs(pend) - 1;
    const unsigned lk = __shfl_sync(FULL, key, ldr);
    const int lR = __shfl_sync(FULL, R, ldr);
    const bool mem = ((pend >> lane) & 1u) && key == lk;
    pend &= ~__ballot_sync(FULL, mem);
    // slot s = 4 k + c (corner k, channel c < 3); lane bits 4, 3, 2, 1 <->
    // slot bits 3 (corner row), 2 (corner column), 1, 0 (channel)
    const float m0 = mem ? w[0] : 0.f, m1 = mem ? w[1] : 0.f, m2 = mem ? w[2] : 0.f, m3 = mem ? w[3] : 0.f;
    const float gc[3] = {g.x, g.y, g.z};
    float a[8];  // after step 1: slot 4 k' + c of corner row (u16 ? 1 : 0)
    {
      const float wk0 = u16 ? m2 : m0, wk1 = u16 ? m3 : m1, ws0 = u16 ? m0 : m2, ws1 = u16 ? m1 : m3;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        a[c] = fmaf(wk0, gc[c], __shfl_xor_sync(FULL, ws0 * gc[c], 16));
        a[4 + c] = fmaf(wk1, gc[c], __shfl_xor_sync(FULL, ws1 * gc[c], 16));
      }
      a[3] = a[7] = 0.f;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {  // corner column
      const float snd = u8 ? a[c] : a[4 + c], kp = u8 ? a[4 + c] : a[c];
      a[c] = kp + __shfl_xor_sync(FULL, snd, 8);
    }
    a[3] = 0.f;
#pragma unroll
    for (int c = 0; c < 2; ++c) {  // channel bit 1
      const float snd = u4 ? a[c] : a[2 + c], kp = u4 ? a[2 + c] : a[c];
      a[c] = kp + __shfl_xor_sync(FULL, snd, 4);
    }
    {  // channel bit 0
      const float snd = u2 ? a[0] : a[1], kp = u2 ? a[1] : a[0];
      a[0] = kp + __shfl_xor_sync(FULL, snd, 2);
    }
    a[0] += __shfl_xor_sync(FULL, a[0], 1);
    const int sl = lane >> 1, c = sl & 3, k = sl >> 2;
    if (!(lane & 1) && c < 3) {
      const unsigned lt0 = (lk >> 2) & ((1u << 25) - 1u);
      const unsigned ldx = (lk >> 1) & 1u, ldy = lk & 1u;
      float* p = tg.base((int)(lk >> 27)) + 3 * (lt0 + ((k & 1) ? ldx : 0u) + ((k & 2) ? ldy * (unsigned)lR : 0u)) + c;
      if (tg.smem)
        atomicAdd(p, a[0]);
      else
        red_add(p, a[0]);
    }
  }
}

// IND: the views blended per-splat indirect light (mixed by the visibility);
// a separate instance so the plain path keeps its register budget.
template <bool IND>
__global__ void __launch_bounds__(SB_THREADS, 1) k_shade_bwd(ViewTable vt, long long n_pix, float4* __restrict__ gxa,
                                                             GradTable g, EnvGradLayout lay, int use_smem) {
  extern __shared__ float s_env[];
  const bool want_env = (g.irr != nullptr) || (g.spec[0] != nullptr);
  const bool shared = use_smem && want_env;
  if (shared) {
    for (int i = threadIdx.x; i < lay.total; i += blockDim.x) s_env[i] = 0.f;
    __syncthreads();
  }
  const int L = vt.v[0].env.levels;  // all views of a batch share the scene
  EnvTarget tg;
  tg.smem = shared ? s_env : nullptr;
  tg.g = &g;
  tg.lay = &lay;
  tg.levels = L;
  // each CTA takes a contiguous run of pixels (a band of rows): neighbouring
  // pixels reflect similar directions, so a CTA touches few cube texels and
  // its flush below skips the untouched (zero) ones.  The loop is uniform
  // over the CTA; `live` marks the lanes with a pixel.
  const long long per = (n_pix + gridDim.x - 1) / gridDim.x;
  const long long p_end = min(n_pix, per * (blockIdx.x + 1));
  for (long long pb = per * blockIdx.x; pb < p_end; pb += blockDim.x) {
    const long long p = pb + threadIdx.x;
    const bool live = p < p_end;
    EnvGrad eg = {};  // all zero: lanes without a pixel contribute exact zeros to the shuffles
    if (live) {
      // view of this pixel (views are few; linear scan)
      int v = 0;
      long long off = 0;
      while (v + 1 < vt.n_views && off + (long long)vt.v[v].W * vt.v[v].H <= p) {
        off += (long long)vt.v[v].W * vt.v[v].H;
        ++v;
      }
      const ViewDesc& V = vt.v[v];
      const int pix = (int)(p - off);
      const int px = pix % V.W, py = pix / V.W;
      const float xp = (float)px + 0.5f - V.cx, yp = (float)py + 0.5f - V.cy;
      const float4 a = V.gbuf[2 * pix], b = V.gbuf[2 * pix + 1];
      const float X[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
      const float A = V.acc[pix];
      const float3 d = world_ray(V, xp, yp);
      const float4 dl = V.dl[pix];
      float gX[8], gA;
      if (IND) {
        const float4 xi = V.gind[pix];
        const float ind[3] = {xi.x, xi.y, xi.z};
        float gind[3];
        shade_pixel_bwd(V.env, X, A, d, dl, gX, gA, eg, ind, V.vis ? V.vis[pix] : 1.f, gind);
        V.gxind[pix] = make_float4(gind[0], gind[1], gind[2], 0.f);
      } else {
        shade_pixel_bwd(V.env, X, A, d, dl, gX, gA, eg);
      }
      float gZ = 0.f;
      if (V.gnorm) {  // the depth-normal loss of this view (ts_normal_loss)
        const float4 gn = V.gnorm[pix];
        gX[5] += gn.x;
        gX[6] += gn.y;
        gX[7] += gn.z;
        gA += gn.w;
        gZ = V.gzsum[pix];
      }
      gxa[3 * p] = make_float4(gX[0], gX[1], gX[2], gX[3]);
      gxa[3 * p + 1] = make_float4(gX[4], gX[5], gX[6], gX[7]);
      gxa[3 * p + 2] = make_float4(gA, gZ, 0.f, 0.f);
    }
    if (want_env) {
      const EnvDesc& E = vt.v[0].env;
      const bool ok = live && eg.ok;
      const int l0 = ok ? eg.l0 : 0, l1 = ok ? eg.l1 : 0;
      if (g.spec[0]) {
        warp_cell_scatter(tg, ok, l0, E.spec_res[l0], eg.face_r, eg.b0, eg.gsp, eg.w0);
        if (L > 1) warp_cell_scatter(tg, ok, l1, E.spec_res[l1], eg.face_r, eg.b1, eg.gsp, eg.w1);
      }
      if (g.irr) warp_cell_scatter(tg, ok, L, E.irr_res, eg.face_n, eg.bi, eg.gir, 1.f);
    }
  }
  if (shared) {
    __syncthreads();
    const int nlev = vt.v[0].env.levels;
    for (int i = threadIdx.x; i < lay.total; i += blockDim.x) {
      const float val = s_env[i];
      if (val == 0.f) continue;
      if (i >= lay.irr_off) {
        if (g.irr) red_add(g.irr + (i - lay.irr_off), val);
      } else {
        int l = 0;
        while (l + 1 < nlev && lay.off[l + 1] <= i) ++l;
        if (g.spec[l]) red_add(g.spec[l] + (i - lay.off[l]), val);
      }
    }
  }
}

void launch_shade_bwd(const ViewTable& vt, float4* gxa, const GradTable& g, cudaStream_t st) {
  long long n_pix = 0;
  for (int i = 0; i < vt.n_views; ++i) n_pix += (long long)vt.v[i].W * vt.v[i].H;
  if (n_pix == 0) return;
  // all views of one backward share the scene, hence the environment layout
  const EnvDesc& E = vt.v[0].env;
  EnvGradLayout lay;
  int tot = 0;
  for (int l = 0; l < E.levels; ++l) {
    lay.off[l] = tot;
    tot += 6 * E.spec_res[l] * E.spec_res[l] * 3;
  }
  lay.irr_off = tot;
  tot += 6 * E.irr_res * E.irr_res * 3;
  lay.total = tot;
  const int use_smem = tot <= SB_MAX_SMEM_FLOATS ? 1 : 0;
  const size_t smem = use_smem ? (size_t)tot * sizeof(float) : 0;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  // the shared-memory opt-in is a per-device attribute of the function
  static std::atomic<bool> attr_set[64];
  if (dev < 0 || dev >= 64 || !attr_set[dev].load()) {
    cudaFuncSetAttribute(k_shade_bwd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SB_MAX_SMEM_FLOATS * 4);
    cudaFuncSetAttribute(k_shade_bwd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SB_MAX_SMEM_FLOATS * 4);
    if (dev >= 0 && dev < 64) attr_set[dev].store(true);
  }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long want = (n_pix + SB_THREADS - 1) / SB_THREADS;
  const int per_sm = use_smem ? 1 : 4;
  const int grid = (int)((want < (long long)sms * per_sm) ? want : (long long)sms * per_sm);
  // a batch's views are all rendered with or all without indirect light
  if (vt.v[0].gind && vt.v[0].gxind)
    k_shade_bwd<true><<<grid, SB_THREADS, smem, st>>>(vt, n_pix, gxa, g, lay, use_smem);
  else
    k_shade_bwd<false><<<grid, SB_THREADS, smem, st>>>(vt, n_pix, gxa, g, lay, use_smem);
  note_launches(1);
}

}  // namespace ts
