// Shared device-side definitions of the textured 2DGS renderer (sm_103a).
//
// Layout decisions (HBM-resident, 16-byte aligned for vector loads):
//   splat means / quaternions: float4 per splat (means padded with 0)
//   scales: float2, opacity: float
//   texels: [n][T][T][8] in float32 (32 B / texel) or bf16/f16 (16 B / texel)
//   per-item raster record: 5 x float4 = 80 B (see Record below)
//   pairs: (global tile id u32, item id u32) as two planes
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace ts {

constexpr int TILE = 16;
constexpr int TILE_PIX = TILE * TILE;
constexpr int MAX_VIEWS = 32;
constexpr int MAX_LEVELS = 12;
constexpr int NCH = 8;

// Thresholds of the method, as float32 values (identical in the oracle).
__host__ __device__ constexpr float kNear() { return 0.2f; }
__host__ __device__ constexpr float kAlphaMin() { return 1.0f / 255.0f; }
__host__ __device__ constexpr float kAlphaMax() { return 0.99f; }
__host__ __device__ constexpr float kTMin() { return 1e-4f; }
__host__ __device__ constexpr float kAMin() { return 1e-7f; }
__host__ __device__ constexpr float kNdotVMin() { return 1e-4f; }

// Per-item record gradients summed by the backward rasteriser (float64):
// 0-8 d/d(h_u, h_v, h_w), 9 d/do, 10-12 the torque of the normal-mapping
// frame, 13 d/dD (through the depth channel); stride 14 keeps rows 16-byte
// aligned.
constexpr int kRecGrads = 14;
constexpr int kRecGradStride = 14;

enum Dtype : int { DT_F32 = 0, DT_BF16 = 1, DT_F16 = 2 };

// Words of the per-device sort error flags (see sort_error_flag).
enum SortFlag : int { SORT_FLAG_LISTS = 0, SORT_FLAG_ORDER = 1 };

// Texture sampler of the forward rasteriser.
//   SMP_SOFTWARE: bilinear filter (Eq. 6) in FP32 from the per-splat chart layout;
//   SMP_HW_ATLAS: tex2D on 2-D hardware-texture atlases (supplementary Sec. 1);
//   SMP_FLAT:     one attribute vector per splat (texel (0, 0) of its chart), no
//                 texture lookup -- the untextured baseline of the paper's Table 3.
enum Sampler : int { SMP_SOFTWARE = 0, SMP_HW_ATLAS = 1, SMP_FLAT = 2 };

// Optional features of a render, as template bits of the rasterisers:
//   FEAT_IND: per-splat SH indirect light blended into its own channel and
//             mixed with the environment by the visibility (Eq. 9, Eq. 12);
//   FEAT_N2:  two-component tangent normals (Sec. 3.5.1): channels 5-6 hold
//             (n_x, n_y), n_z = sqrt(max(0, 1 - n_x^2 - n_y^2)) is rebuilt
//             from the interpolated pair and channel 7 is not read.
enum Feature : int { FEAT_IND = 1, FEAT_N2 = 2 };

// Environment light (Eq. 11-12): specular mip chain, irradiance cube, BRDF LUT.
struct EnvDesc {
  const void* spec[MAX_LEVELS];  // [6][R_l][R_l][3]
  int spec_res[MAX_LEVELS];
  int levels;
  const void* irr;  // [6][R][R][3]
  int irr_res;
  int cube_dtype;   // DT_F32 or DT_F16
  const float* lut; // [R][R][2]
  int lut_res;
};

// One view of a batch: camera, output buffers and the scene it renders.
struct ViewDesc {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  int W, H, tiles_x, tiles_y;
  int tile_off;   // first global tile of the view
  int item_off;   // first item (view-local splat index 0 maps here)
  int pix_off;    // first pixel of the view in batch-wide per-pixel buffers
  int n_splats;
  // scene
  const float4* means;
  const float4* quats;
  const float2* scales;
  const float* opacity;
  const void* texels;
  int T;
  int tex_dtype;
  int tex_v8;     // float32 texels at a 32-byte aligned base: one 32-byte load per texel
  // 2-D atlases for SMP_HW_ATLAS: channels 0-3 and 4-7, and each splat's
  // chart origin (texels) -- the indirection buffer of supplementary Sec. 1
  cudaTextureObject_t atlas2d[2];
  const uint2* chart;
  // indirect light: per-splat SH coefficients (degree sh_deg <= 2, K = (deg+1)^2
  // basis functions x RGB, rows of sh_stride floats), NULL when the scene has
  // none; the view's visibility V [H][W] (NULL: V = 1)
  const float* sh;
  int sh_deg, sh_stride;
  const float* vis;
  EnvDesc env;
  // outputs / saved state
  float4* rgba;   // [H][W]
  float4* gbuf;   // [H][W][2] (X of Eq. 9, 8 channels)
  float* trans;   // [H][W]
  float* acc;     // [H][W] blended coverage A = sum alpha_i T_i (not 1 - T: no cancellation)
  float* zsum;    // [H][W] blended camera depth of the hits, sum alpha_i T_i z_i (saved renders)
  float4* gind;   // [H][W] blended indirect light X_ind (xyz), saved when the batch has SH
  float4* gxind;  // [H][W] backward scratch: dL/dX_ind (xyz)
  const float4* gnorm;  // [H][W] extra dL/dN (xyz), dL/dA (w) from the depth-normal loss, or NULL
  const float* gzsum;   // [H][W] dL/d zsum from the depth-normal loss, or NULL
  int* last;      // [H][W]
  const float4* dl;  // backward input dL/drgba [H][W]
};

struct ViewTable {
  int n_views;
  int n_tiles;   // total tiles
  int n_items;   // total items
  // the rasterisers' tiles in launch order (CTA b takes tile tile_order[b]),
  // or NULL for tile order
  const uint32_t* tile_order;
  // the sort error flags (two words, see SortFlag), or NULL
  const int* sort_err;
  ViewDesc v[MAX_VIEWS];
};

// Raster record of one (view, splat) item, written by the preprocess.
// h_u, h_v, h_w are the homography rows of the splat in centred pixel
// coordinates (x' = x + 0.5 - cx, y' = y + 0.5 - cy): u = h_u.x / h_w.x,
// v = h_v.x / h_w.x with x = (x', y', 1) (closed-form ray-splat
// intersection, Sec. 3.1).  tu, tv, nf: world-space tangent frame with the
// normal turned towards the camera (for normal mapping, Eq. 7).  The h_u and
// h_v coefficients are interleaved so that (u, v) numerators evaluate as
// channel pairs from adjacent registers.  D = p_c . n_c (camera space) makes
// the camera depth of the hit z = D / (h_w . x) (Eq. 1: the ray meets the
// splat plane).  The splat of an item is item - item_off of its view.
struct Record {
  float4 r0;  // hu0 hv0 hu1 hv1
  float4 r1;  // hu2 hv2 hw0 hw1
  float4 r2;  // hw2 opacity tu0 tu1
  float4 r3;  // tu2 tv0 tv1 tv2
  float4 r4;  // nf0 nf1 nf2 D
};
static_assert(sizeof(Record) == 80, "record is 5 x 16 B");

__device__ __forceinline__ int find_view(const ViewTable& vt, int tile) {
  int v = 0;
  while (v + 1 < vt.n_views && vt.v[v + 1].tile_off <= tile) ++v;
  return v;
}
__device__ __forceinline__ int find_view_item(const ViewTable& vt, int item) {
  int v = 0;
  while (v + 1 < vt.n_views && vt.v[v + 1].item_off <= item) ++v;
  return v;
}

// ---- paired FP32 (sm_100+ float2 ops) -----------------------------------------
// One instruction for two lanes of arithmetic; per component the rounding is
// that of the scalar fmaf / __fmul_rn / __fadd_rn, so a paired expression gives
// bit-identical results to the same scalar expression.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// ---- texel loads (stored dtype -> float32) ----------------------------------
// One float32 texel (8 channels, 32 bytes) in a single 256-bit load; p must
// be 32-byte aligned (callers check the atlas base once per view).
__device__ __forceinline__ void load_texel_v8(const float* p, float out[8]) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(out[0]), "=f"(out[1]), "=f"(out[2]), "=f"(out[3]), "=f"(out[4]), "=f"(out[5]), "=f"(out[6]),
        "=f"(out[7])
      : "l"(p));
}

// The same, kept in program order relative to the other ordered loads
// (volatile): callers that consume texels in phases keep fewer live.
__device__ __forceinline__ void load_texel_v8_ordered(const float* p, float out[8]) {
  asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(out[0]), "=f"(out[1]), "=f"(out[2]), "=f"(out[3]), "=f"(out[4]), "=f"(out[5]), "=f"(out[6]),
                 "=f"(out[7])
               : "l"(p));
}

__device__ __forceinline__ void load_texel(const void* base, int dtype, long long idx, float out[8]) {
  if (dtype == DT_F32) {
    const float4* p = reinterpret_cast<const float4*>(base) + idx * 2;
    float4 a = __ldg(p), b = __ldg(p + 1);
    out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
    out[4] = b.x; out[5] = b.y; out[6] = b.z; out[7] = b.w;
  } else {
    uint4 raw = __ldg(reinterpret_cast<const uint4*>(base) + idx);
    uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (dtype == DT_BF16) {
        out[2 * i] = __uint_as_float(w[i] << 16);
        out[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
      } else {
        __half2 h = *reinterpret_cast<__half2*>(&w[i]);
        float2 f = __half22float2(h);
        out[2 * i] = f.x;
        out[2 * i + 1] = f.y;
      }
    }
  }
}

__device__ __forceinline__ float3 load_cube3(const void* base, int dtype, long long idx) {
  if (dtype == DT_F32) {
    const float* p = reinterpret_cast<const float*>(base) + idx * 3;
    return make_float3(__ldg(p), __ldg(p + 1), __ldg(p + 2));
  }
  const __half* p = reinterpret_cast<const __half*>(base) + idx * 3;
  return make_float3(__half2float(p[0]), __half2float(p[1]), __half2float(p[2]));
}

// Vector reduction into global memory (sm_90+ red.global.add.v4.f32).
__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c),
               "f"(d)
               : "memory");
}
__device__ __forceinline__ void red_add(float* addr, float a) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(addr), "f"(a) : "memory");
}

}  // namespace ts
