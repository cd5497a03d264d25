// Optimizer step for training (Sec. 3.6 optimises splats, textures and the
// environment end to end): Adam on float32 master parameters, fused with
// zeroing the consumed gradient and writing the stored copy (float32, or
// bfloat16 / float16 rounded to nearest even) that the renderer reads.
// One pass over 4 x 16-byte streams per element group; HBM-bound.
#include "kernels.h"
#include "prof.h"

namespace ts {

template <int SD>
__global__ void __launch_bounds__(256) k_adam(float* __restrict__ p, float* __restrict__ g, float* __restrict__ m,
                                              float* __restrict__ v, long long n, float lr, float b1, float b2,
                                              float eps, float bc1, float bc2, void* __restrict__ shadow,
                                              int zero_grad) {
  const long long n4 = n >> 2;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    float4 pp = reinterpret_cast<float4*>(p)[i];
    const float4 gg = reinterpret_cast<const float4*>(g)[i];
    float4 mm = reinterpret_cast<float4*>(m)[i];
    float4 vv = reinterpret_cast<float4*>(v)[i];
    float* pa = &pp.x;
    const float* ga = &gg.x;
    float* ma = &mm.x;
    float* va = &vv.x;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ma[k] = fmaf(b1, ma[k], (1.f - b1) * ga[k]);
      va[k] = fmaf(b2, va[k], (1.f - b2) * ga[k] * ga[k]);
      const float mh = ma[k] * bc1, vh = va[k] * bc2;
      pa[k] -= lr * mh / (sqrtf(vh) + eps);
    }
    reinterpret_cast<float4*>(p)[i] = pp;
    reinterpret_cast<float4*>(m)[i] = mm;
    reinterpret_cast<float4*>(v)[i] = vv;
    if (zero_grad) reinterpret_cast<float4*>(g)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (SD == DT_F32) {
      reinterpret_cast<float4*>(shadow)[i] = pp;
    } else if (SD == DT_BF16) {
      __nv_bfloat162 a = __floats2bfloat162_rn(pp.x, pp.y), b = __floats2bfloat162_rn(pp.z, pp.w);
      uint2 w;
      w.x = *reinterpret_cast<uint32_t*>(&a);
      w.y = *reinterpret_cast<uint32_t*>(&b);
      reinterpret_cast<uint2*>(shadow)[i] = w;
    } else if (SD == DT_F16) {
      __half2 a = __floats2half2_rn(pp.x, pp.y), b = __floats2half2_rn(pp.z, pp.w);
      uint2 w;
      w.x = *reinterpret_cast<uint32_t*>(&a);
      w.y = *reinterpret_cast<uint32_t*>(&b);
      reinterpret_cast<uint2*>(shadow)[i] = w;
    }
  }
  // tail (n not a multiple of 4), handled by the first threads
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long j = (n4 << 2) + t;
  if (t < 4 && j < n) {
    const float gj = g[j];
    m[j] = fmaf(b1, m[j], (1.f - b1) * gj);
    v[j] = fmaf(b2, v[j], (1.f - b2) * gj * gj);
    p[j] -= lr * (m[j] * bc1) / (sqrtf(v[j] * bc2) + eps);
    if (zero_grad) g[j] = 0.f;
    if (SD == DT_F32) reinterpret_cast<float*>(shadow)[j] = p[j];
    else if (SD == DT_BF16) reinterpret_cast<__nv_bfloat16*>(shadow)[j] = __float2bfloat16_rn(p[j]);
    else if (SD == DT_F16) reinterpret_cast<__half*>(shadow)[j] = __float2half_rn(p[j]);
  }
}

void launch_adam(float* p, float* g, float* m, float* v, long long n, float lr, float b1, float b2, float eps,
                 long long step, void* shadow, int shadow_dtype, int zero_grad, cudaStream_t st) {
  if (n <= 0) return;
  const float bc1 = (float)(1.0 / (1.0 - pow((double)b1, (double)step)));
  const float bc2 = (float)(1.0 / (1.0 - pow((double)b2, (double)step)));
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long n4 = (n + 3) >> 2;
  const long long want = (n4 + 255) / 256;
  const int grid = (int)(want < (long long)sms * 8 ? want : (long long)sms * 8);
  if (!shadow)
    k_adam<-1><<<grid, 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, bc1, bc2, shadow, zero_grad);
  else if (shadow_dtype == DT_F32)
    k_adam<DT_F32><<<grid, 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, bc1, bc2, shadow, zero_grad);
  else if (shadow_dtype == DT_BF16)
    k_adam<DT_BF16><<<grid, 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, bc1, bc2, shadow, zero_grad);
  else
    k_adam<DT_F16><<<grid, 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, bc1, bc2, shadow, zero_grad);
  note_launches(1);
}

}  // namespace ts
