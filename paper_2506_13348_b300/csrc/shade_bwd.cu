// Shading adjoint (Eq. 10-12) as its own pass over all pixels of a batch.
//
// Each pixel turns dL/drgba into dL/dX (8 G-buffer channels) and dL/dA,
// written for the backward rasteriser (3 x float4 per pixel), and scatters
// its gradient into the environment maps with bilinear / trilinear weights.
// Environment maps are small and every pixel of a view hits them, so
// global atomics on them contend heavily; when all levels and the irradiance
// cube fit (<= 96 KB of float32 gradients) each CTA accumulates them in
// shared memory and adds its copy to the global gradient once at the end
// (persistent grid, a few CTAs per SM).
#include "kernels.h"
#include "prof.h"
#include "shading.cuh"

namespace ts {

constexpr int SB_THREADS = 256;
constexpr int SB_MAX_SMEM_FLOATS = 24 * 1024;  // 96 KB

// Offsets of each level / the irradiance cube inside one flat gradient array.
struct EnvGradLayout {
  int off[MAX_LEVELS];
  int irr_off;
  int total;
};

__device__ __forceinline__ void scatter_cube(float* dst, int R, int face, const Bil& b, float3 g, float scale,
                                             bool shared) {
  const int fb = face * R * R;
  const float gx = 1.f - b.fx, gy = 1.f - b.fy;
  const float w[4] = {gx * gy * scale, b.fx * gy * scale, gx * b.fy * scale, b.fx * b.fy * scale};
  const int idx[4] = {fb + b.ja * R + b.ia, fb + b.ja * R + b.ib, fb + b.jb * R + b.ia, fb + b.jb * R + b.ib};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (w[k] == 0.f) continue;
    float* p = dst + idx[k] * 3;
    if (shared) {
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

// Environment part of the adjoint: recomputes the lookups and scatters.
__device__ __forceinline__ void env_scatter(const EnvDesc& E, const float X[8], float A, float3 d, float4 g,
                                            float* const* spec_dst, float* irr_dst, bool shared) {
  ShadeState s;
  shade_pixel(E, X, A, d, &s);
  if (!s.ok) return;
  const float inv_pi = 0.318309886183790672f;
  float3 gsp, gir;
  {
    const float gc[3] = {g.x, g.y, g.z};
    float v1[3], v2[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float gLo = A * gc[c];
      v1[c] = (s.F0[c] * s.lt.x + s.lt.y) * gLo;
      v2[c] = s.lam[c] * inv_pi * (1.f - s.met) * gLo;
    }
    gsp = make_float3(v1[0], v1[1], v1[2]);
    gir = make_float3(v2[0], v2[1], v2[2]);
  }
  const CubeCoord cr = cube_coord(s.wr);
  Bil b;
  b = bil_setup(cr.s * E.spec_res[s.l0] - 0.5f, cr.t * E.spec_res[s.l0] - 0.5f, E.spec_res[s.l0], E.spec_res[s.l0]);
  const float w0 = (E.levels > 1) ? (1.f - s.f) : 1.f;
  scatter_cube(spec_dst[s.l0], E.spec_res[s.l0], cr.face, b, gsp, w0, shared);
  if (E.levels > 1) {
    b = bil_setup(cr.s * E.spec_res[s.l1] - 0.5f, cr.t * E.spec_res[s.l1] - 0.5f, E.spec_res[s.l1],
                  E.spec_res[s.l1]);
    scatter_cube(spec_dst[s.l1], E.spec_res[s.l1], cr.face, b, gsp, s.f, shared);
  }
  const CubeCoord cn = cube_coord(s.Nh);
  b = bil_setup(cn.s * E.irr_res - 0.5f, cn.t * E.irr_res - 0.5f, E.irr_res, E.irr_res);
  scatter_cube(irr_dst, E.irr_res, cn.face, b, gir, 1.f, shared);
}

__global__ void __launch_bounds__(SB_THREADS) k_shade_bwd(ViewTable vt, long long n_pix, float4* __restrict__ gxa,
                                                          GradTable g, EnvGradLayout lay, int use_smem) {
  extern __shared__ float s_env[];
  const bool want_env = (g.irr != nullptr) || (g.spec[0] != nullptr);
  const bool shared = use_smem && want_env;
  if (shared) {
    for (int i = threadIdx.x; i < lay.total; i += blockDim.x) s_env[i] = 0.f;
    __syncthreads();
  }
  // each CTA takes a contiguous run of pixels (a band of rows): neighbouring
  // pixels reflect similar directions, so a CTA touches few cube texels and
  // its flush below skips the untouched (zero) ones
  const long long per = (n_pix + gridDim.x - 1) / gridDim.x;
  const long long p_end = min(n_pix, per * (blockIdx.x + 1));
  for (long long p = per * blockIdx.x + threadIdx.x; p < p_end; p += blockDim.x) {
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
    shade_pixel_bwd(V.env, X, A, d, dl, gX, gA, nullptr, nullptr);
    gxa[3 * p] = make_float4(gX[0], gX[1], gX[2], gX[3]);
    gxa[3 * p + 1] = make_float4(gX[4], gX[5], gX[6], gX[7]);
    gxa[3 * p + 2] = make_float4(gA, 0.f, 0.f, 0.f);
    if (want_env) {
      if (shared) {
        float* sp[MAX_LEVELS];
        for (int l = 0; l < V.env.levels; ++l) sp[l] = s_env + lay.off[l];
        env_scatter(V.env, X, A, d, dl, sp, s_env + lay.irr_off, true);
      } else {
        env_scatter(V.env, X, A, d, dl, g.spec, g.irr, false);
      }
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
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_shade_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, SB_MAX_SMEM_FLOATS * 4);
    attr_set = true;
  }
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long want = (n_pix + SB_THREADS - 1) / SB_THREADS;
  const int per_sm = use_smem ? 2 : 8;
  const int grid = (int)((want < (long long)sms * per_sm) ? want : (long long)sms * per_sm);
  k_shade_bwd<<<grid, SB_THREADS, smem, st>>>(vt, n_pix, gxa, g, lay, use_smem);
  note_launches(1);
}

}  // namespace ts
