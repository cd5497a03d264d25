// Upload-time packing and the L1 image loss.
#include <algorithm>
#include "kernels.h"
#include "prof.h"

namespace ts {

// Atlas pack: float32 texels -> stored dtype, round to nearest even.
__global__ void k_pack_texels(const float* __restrict__ src, void* __restrict__ dst, long long n, int dtype) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float x = src[i];
  if (dtype == DT_F32) {
    reinterpret_cast<float*>(dst)[i] = x;
  } else if (dtype == DT_BF16) {
    reinterpret_cast<__nv_bfloat16*>(dst)[i] = __float2bfloat16_rn(x);
  } else {
    reinterpret_cast<__half*>(dst)[i] = __float2half_rn(x);
  }
}

// Same, eight elements (one texel) per step: two 16-byte loads, one 16-byte
// store (bf16 / f16) -- HBM-bound, grid-stride over a grid sized to the SMs.
template <int DT>
__global__ void __launch_bounds__(256) k_pack_texels8(const float4* __restrict__ src, uint4* __restrict__ dst,
                                                      long long n8) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n8; i += (long long)gridDim.x * blockDim.x) {
    const float4 a = __ldcs(src + 2 * i), b = __ldcs(src + 2 * i + 1);
    uint4 o;
    if (DT == DT_BF16) {
      const __nv_bfloat162 p0 = __floats2bfloat162_rn(a.x, a.y), p1 = __floats2bfloat162_rn(a.z, a.w);
      const __nv_bfloat162 p2 = __floats2bfloat162_rn(b.x, b.y), p3 = __floats2bfloat162_rn(b.z, b.w);
      o = make_uint4(*reinterpret_cast<const uint32_t*>(&p0), *reinterpret_cast<const uint32_t*>(&p1),
                     *reinterpret_cast<const uint32_t*>(&p2), *reinterpret_cast<const uint32_t*>(&p3));
    } else {
      const __half2 p0 = __floats2half2_rn(a.x, a.y), p1 = __floats2half2_rn(a.z, a.w);
      const __half2 p2 = __floats2half2_rn(b.x, b.y), p3 = __floats2half2_rn(b.z, b.w);
      o = make_uint4(*reinterpret_cast<const uint32_t*>(&p0), *reinterpret_cast<const uint32_t*>(&p1),
                     *reinterpret_cast<const uint32_t*>(&p2), *reinterpret_cast<const uint32_t*>(&p3));
    }
    dst[i] = o;
  }
}

void launch_pack_texels(const float* src, void* dst, long long n, int dtype, cudaStream_t st) {
  if (n <= 0) return;
  const bool vec = dtype != DT_F32 && n % 8 == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(dst) & 15) == 0;
  if (vec) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long n8 = n / 8;
    const long long want = (n8 + 255) / 256;
    const unsigned grid = (unsigned)(want < (long long)sms * 8 ? want : (long long)sms * 8);
    if (dtype == DT_BF16)
      k_pack_texels8<DT_BF16><<<grid, 256, 0, st>>>(reinterpret_cast<const float4*>(src), reinterpret_cast<uint4*>(dst), n8);
    else
      k_pack_texels8<DT_F16><<<grid, 256, 0, st>>>(reinterpret_cast<const float4*>(src), reinterpret_cast<uint4*>(dst), n8);
  } else {
    k_pack_texels<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, n, dtype);
  }
  note_launches(1);
}

void launch_pack_f16(const float* src, __half* dst, long long n, cudaStream_t st) {
  launch_pack_texels(src, dst, n, DT_F16, st);
}

__global__ void k_pad4(const float* __restrict__ src, int comps, float4* __restrict__ dst, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float v[4] = {0.f, 0.f, 0.f, 0.f};
  for (int c = 0; c < comps; ++c) v[c] = src[i * comps + c];
  dst[i] = make_float4(v[0], v[1], v[2], v[3]);
}

void launch_pad4(const float* src, int comps, float4* dst, long long n, cudaStream_t st) {
  if (n > 0) {
    k_pad4<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, comps, dst, n);
    note_launches(1);
  }
}

// Upload check of the splat parameters the renderer divides by or
// normalises: finite centres, a quaternion with finite components and a
// squared norm of at least 1e-20 (it is normalised), finite scales > 0
// (the intersection divides by them), opacity in [0, 1].  out[0] counts the
// bad splats, out[1] is the smallest bad index, out[2] ORs the reasons
// (1 centre, 2 quaternion, 4 scale, 8 opacity).
__global__ void k_validate_gaussians(const float4* __restrict__ means, const float4* __restrict__ quats,
                                     const float2* __restrict__ scales, const float* __restrict__ opac, long long n,
                                     unsigned* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float4 p = means[i], q = quats[i];
    const float2 s = scales[i];
    const float o = opac[i];
    unsigned why = 0;
    if (!(isfinite(p.x) && isfinite(p.y) && isfinite(p.z))) why |= 1u;
    const float q2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
    if (!(isfinite(q.x) && isfinite(q.y) && isfinite(q.z) && isfinite(q.w)) || !(q2 >= 1e-20f)) why |= 2u;
    if (!(isfinite(s.x) && isfinite(s.y) && s.x > 0.f && s.y > 0.f)) why |= 4u;
    if (!(o >= 0.f && o <= 1.f)) why |= 8u;
    if (why) {
      atomicAdd(out, 1u);
      atomicMin(out + 1, (unsigned)min(i, 0xfffffffell));
      atomicOr(out + 2, why);
    }
  }
}

void launch_validate_gaussians(const float4* means, const float4* quats, const float2* scales, const float* opac,
                               long long n, unsigned* out, cudaStream_t st) {
  if (n > 0) {
    const unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 148 * 8);
    k_validate_gaussians<<<blocks, 256, 0, st>>>(means, quats, scales, opac, n, out);
    note_launches(1);
  }
}

// Totals of the statistics pass's texel bitmap: set bits (distinct texels
// read by blended fragments) and items with any bit set (distinct splats
// blended at some pixel).  One warp per item, grid-stride.
__global__ void k_touch_counts(const uint32_t* __restrict__ touched, long long n_items, int wpi,
                               unsigned long long* __restrict__ counts) {
  const int lane = threadIdx.x & 31;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  unsigned long long bits = 0, items = 0;
  for (long long i = w0; i < n_items; i += nw) {
    unsigned c = 0;
    for (int k = lane; k < wpi; k += 32) c += __popc(touched[i * wpi + k]);
    c = __reduce_add_sync(0xffffffffu, c);
    bits += c;
    items += c != 0;
  }
  if (lane == 0 && (bits | items)) {
    atomicAdd(counts + 2, bits);
    atomicAdd(counts + 3, items);
  }
}

void launch_touch_counts(const uint32_t* touched, long long n_items, int words_per_item, unsigned long long* counts,
                         cudaStream_t st) {
  if (n_items > 0) {
    const unsigned blocks = (unsigned)std::min<long long>((n_items + 7) / 8, 148 * 8);
    k_touch_counts<<<blocks, 256, 0, st>>>(touched, n_items, words_per_item, counts);
    note_launches(1);
  }
}

// Activations of the raw optimisation variables: s = exp(log s) per scale
// component, o = sigmoid(logit o) (the 3DGS / 2DGS parameterisation the
// optimisation of Sec. 3.6 runs on).  Element i < 2n is a scale component,
// 2n <= i < 3n an opacity.
__global__ void k_activate(const float* __restrict__ log_s, const float* __restrict__ logit_o, long long n,
                           float* __restrict__ s, float* __restrict__ o) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 2 * n) {
    s[i] = expf(log_s[i]);
  } else if (i < 3 * n) {
    const long long k = i - 2 * n;
    o[k] = 1.f / (1.f + expf(-logit_o[k]));
  }
}

// Chain rule of k_activate: dL/dlog s = dL/ds s, dL/dlogit o = dL/do o (1 - o).
__global__ void k_activate_bwd(const float* __restrict__ s, const float* __restrict__ o,
                               const float* __restrict__ gs, const float* __restrict__ go, long long n,
                               float* __restrict__ g_log_s, float* __restrict__ g_logit_o, int accumulate) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 2 * n) {
    const float v = gs[i] * s[i];
    g_log_s[i] = accumulate ? g_log_s[i] + v : v;
  } else if (i < 3 * n) {
    const long long k = i - 2 * n;
    const float v = go[k] * o[k] * (1.f - o[k]);
    g_logit_o[k] = accumulate ? g_logit_o[k] + v : v;
  }
}

void launch_activate(const float* log_s, const float* logit_o, long long n, float* s, float* o, cudaStream_t st) {
  if (n > 0) {
    k_activate<<<(unsigned)((3 * n + 255) / 256), 256, 0, st>>>(log_s, logit_o, n, s, o);
    note_launches(1);
  }
}

void launch_activate_bwd(const float* s, const float* o, const float* gs, const float* go, long long n,
                         float* g_log_s, float* g_logit_o, int accumulate, cudaStream_t st) {
  if (n > 0) {
    k_activate_bwd<<<(unsigned)((3 * n + 255) / 256), 256, 0, st>>>(s, o, gs, go, n, g_log_s, g_logit_o, accumulate);
    note_launches(1);
  }
}

// L1 over RGB: loss = mean |rgb - target|, dL/drgb = sign / (3 n), dL/dalpha = 0.
// Grid-stride over pixels; one atomic per block (a single float receives
// the loss, so per-warp atomics would serialise on it).
constexpr int L1_THREADS = 256;

__global__ void __launch_bounds__(L1_THREADS) k_l1_loss(const float4* __restrict__ rgba,
                                                         const float4* __restrict__ tgt, long long n,
                                                         float* __restrict__ loss, float4* __restrict__ grad) {
  __shared__ float s_part[L1_THREADS / 32];
  const float k = 1.f / (3.f * (float)n);
  auto sgn = [](float d) { return d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f); };
  float s = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float4 a = rgba[i], b = tgt[i];
    const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    s += fabsf(dx) + fabsf(dy) + fabsf(dz);
    grad[i] = make_float4(sgn(dx) * k, sgn(dy) * k, sgn(dz) * k, 0.f);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < L1_THREADS / 32; ++w) t += s_part[w];
    if (t != 0.f) atomicAdd(loss, t * k);
  }
}

void launch_l1_loss(const float4* rgba, const float4* target, long long n, float* loss, float4* grad,
                    cudaStream_t st) {
  cudaMemsetAsync(loss, 0, sizeof(float), st);
  if (n > 0) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (n + L1_THREADS - 1) / L1_THREADS;
    const int grid = (int)(want < (long long)sms * 4 ? want : (long long)sms * 4);
    k_l1_loss<<<grid, L1_THREADS, 0, st>>>(rgba, target, n, loss, grad);
    note_launches(1);
  }
}

}  // namespace ts
