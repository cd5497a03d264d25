// Image term of the training loss (Sec. 3.6): L_img = (1 - lambda) L1 +
// lambda (1 - SSIM) over the RGB channels, with SSIM the structural
// similarity index under an 11x11 Gaussian window (sigma 1.5, zero padding,
// C1 = 0.01^2, C2 = 0.03^2), averaged over pixels and channels.
//
// Two tiled passes over 32x32 output tiles (42x42 inputs with the 5-pixel
// halo in shared memory, separable blur: a horizontal pass into shared
// memory, then a vertical pass per output pixel):
// One CTA per tile and channel.
//   k_ssim_fwd: the five blurred moments per pixel -> SSIM, the L1 and SSIM
//     sums (float64 atomics, one per CTA), and per pixel and channel the
//     loss derivatives w.r.t. the three moments the image enters
//     (mu_x, E[x x], E[x y]), scaled by dL/dSSIM;
//   k_ssim_bwd: blurs those three maps (the adjoint of the zero-padded
//     window sum is the same window sum) and combines them,
//     dL/dx = G*a + 2 x G*b + y G*c, plus the L1 term.
#include <atomic>
#include <cmath>

#include "kernels.h"
#include "prof.h"

namespace ts {

namespace {

constexpr int SS_TO = 32;              // output tile side
constexpr int SS_HALO = 5;             // window radius
constexpr int SS_IN = SS_TO + 2 * SS_HALO;
constexpr int SS_THREADS = 256;
constexpr float SS_C1 = 0.01f * 0.01f;
constexpr float SS_C2 = 0.03f * 0.03f;

__constant__ float c_gauss[11];

__device__ __forceinline__ float chan(const float4& v, int c) { return c == 0 ? v.x : (c == 1 ? v.y : v.z); }

__global__ void __launch_bounds__(SS_THREADS) k_ssim_fwd(const float4* __restrict__ img, const float4* __restrict__ tgt,
                                                         int W, int H, float dLdS, float* __restrict__ part,
                                                         double* __restrict__ acc) {
  __shared__ float sx[SS_IN][SS_IN + 1], sy[SS_IN][SS_IN + 1];
  __shared__ float hs[5][SS_IN][SS_TO];
  __shared__ double red[2][SS_THREADS / 32];
  const int ox = blockIdx.x * SS_TO, oy = blockIdx.y * SS_TO;
  const int tid = threadIdx.x;
  const long long N = (long long)W * H;
  float l1 = 0.f, ss = 0.f;
  const int ch = blockIdx.z;  // one RGB channel per CTA
  {
    for (int i = tid; i < SS_IN * SS_IN; i += SS_THREADS) {
      const int r = i / SS_IN, c = i - r * SS_IN;
      const int gx = ox - SS_HALO + c, gy = oy - SS_HALO + r;
      float a = 0.f, b = 0.f;
      if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
        const long long p = (long long)gy * W + gx;
        a = chan(img[p], ch);
        b = chan(tgt[p], ch);
      }
      sx[r][c] = a;
      sy[r][c] = b;
    }
    __syncthreads();
    for (int i = tid; i < SS_IN * SS_TO; i += SS_THREADS) {
      const int r = i / SS_TO, c = i - r * SS_TO;
      float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int k = 0; k < 11; ++k) {
        const float g = c_gauss[k], a = sx[r][c + k], b = sy[r][c + k];
        m[0] = fmaf(g, a, m[0]);
        m[1] = fmaf(g, b, m[1]);
        m[2] = fmaf(g, a * a, m[2]);
        m[3] = fmaf(g, b * b, m[3]);
        m[4] = fmaf(g, a * b, m[4]);
      }
#pragma unroll
      for (int q = 0; q < 5; ++q) hs[q][r][c] = m[q];
    }
    __syncthreads();
    for (int i = tid; i < SS_TO * SS_TO; i += SS_THREADS) {
      const int r = i / SS_TO, c = i - r * SS_TO;
      const int gx = ox + c, gy = oy + r;
      if (gx >= W || gy >= H) continue;
      float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int k = 0; k < 11; ++k) {
        const float g = c_gauss[k];
#pragma unroll
        for (int q = 0; q < 5; ++q) m[q] = fmaf(g, hs[q][r + k][c], m[q]);
      }
      const float mx = m[0], my = m[1];
      const float sxx = m[2] - mx * mx, syy = m[3] - my * my, sxy = m[4] - mx * my;
      const float A1 = 2.f * mx * my + SS_C1, A2 = 2.f * sxy + SS_C2;
      const float B1 = mx * mx + my * my + SS_C1, B2 = sxx + syy + SS_C2;
      const float S = (A1 * A2) / (B1 * B2);
      ss += S;
      l1 += fabsf(sx[r + SS_HALO][c + SS_HALO] - sy[r + SS_HALO][c + SS_HALO]);
      // dS/dmu_x, dS/dE[xx], dS/dE[xy] (the image x enters only these three)
      const float dmx = S * (2.f * my / A1 - 2.f * my / A2 - 2.f * mx / B1 + 2.f * mx / B2);
      const float dxx = -S / B2;
      const float dxy = 2.f * S / A2;
      const long long p = (long long)gy * W + gx;
      part[(3 * ch + 0) * N + p] = dLdS * dmx;
      part[(3 * ch + 1) * N + p] = dLdS * dxx;
      part[(3 * ch + 2) * N + p] = dLdS * dxy;
    }
    __syncthreads();
  }
  // block sums -> one float64 atomic per CTA and quantity
  double d1 = l1, d2 = ss;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    d1 += __shfl_xor_sync(0xffffffffu, d1, o);
    d2 += __shfl_xor_sync(0xffffffffu, d2, o);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = d1;
    red[1][tid >> 5] = d2;
  }
  __syncthreads();
  if (tid == 0) {
    double t1 = 0.0, t2 = 0.0;
    for (int w = 0; w < SS_THREADS / 32; ++w) {
      t1 += red[0][w];
      t2 += red[1][w];
    }
    atomicAdd(acc, t1);
    atomicAdd(acc + 1, t2);
  }
}

__global__ void __launch_bounds__(SS_THREADS) k_ssim_bwd(const float4* __restrict__ img, const float4* __restrict__ tgt,
                                                         int W, int H, const float* __restrict__ part, float l1w,
                                                         float4* __restrict__ grad) {
  __shared__ float sp[3][SS_IN][SS_IN + 1];
  __shared__ float hs[3][SS_IN][SS_TO];
  const int ox = blockIdx.x * SS_TO, oy = blockIdx.y * SS_TO;
  const int tid = threadIdx.x;
  const long long N = (long long)W * H;
  constexpr int PER = SS_TO * SS_TO / SS_THREADS;  // output pixels per thread
  const int ch = blockIdx.z;  // one RGB channel per CTA
  for (int i = tid; i < SS_IN * SS_IN; i += SS_THREADS) {
    const int r = i / SS_IN, c = i - r * SS_IN;
    const int gx = ox - SS_HALO + c, gy = oy - SS_HALO + r;
    const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
    const long long p = (long long)gy * W + gx;
#pragma unroll
    for (int j = 0; j < 3; ++j) sp[j][r][c] = in ? part[(3 * ch + j) * N + p] : 0.f;
  }
  __syncthreads();
  for (int i = tid; i < SS_IN * SS_TO; i += SS_THREADS) {
    const int r = i / SS_TO, c = i - r * SS_TO;
    float m[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 11; ++k) {
      const float g = c_gauss[k];
#pragma unroll
      for (int j = 0; j < 3; ++j) m[j] = fmaf(g, sp[j][r][c + k], m[j]);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) hs[j][r][c] = m[j];
  }
  __syncthreads();
  float* gout = reinterpret_cast<float*>(grad);
#pragma unroll
  for (int e = 0; e < PER; ++e) {
    const int i = tid + e * SS_THREADS;
    const int r = i / SS_TO, c = i - r * SS_TO;
    const int gx = ox + c, gy = oy + r;
    if (gx >= W || gy >= H) continue;
    float m[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 11; ++k) {
      const float g = c_gauss[k];
#pragma unroll
      for (int j = 0; j < 3; ++j) m[j] = fmaf(g, hs[j][r + k][c], m[j]);
    }
    const long long p = (long long)gy * W + gx;
    const float x = chan(img[p], ch), y = chan(tgt[p], ch);
    const float d = x - y;
    const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
    gout[4 * p + ch] = m[0] + 2.f * x * m[1] + y * m[2] + l1w * sgn;
    if (ch == 0) gout[4 * p + 3] = 0.f;
  }
}

__global__ void k_loss_finish(const double* __restrict__ acc, double n3, float lam, float* __restrict__ loss) {
  loss[0] = (float)((1.0 - lam) * acc[0] / n3 + lam * (1.0 - acc[1] / n3));
}

std::atomic<bool> g_gauss_set[64];

}  // namespace

int set_gauss_window(int device) {
  if (device < 0 || device >= 64) return 1;
  if (g_gauss_set[device]) return 0;
  float g[11];
  double s = 0.0, t[11];
  for (int k = 0; k < 11; ++k) {
    const double r = k - 5.0;
    t[k] = std::exp(-(r * r) / (2.0 * 1.5 * 1.5));
    s += t[k];
  }
  for (int k = 0; k < 11; ++k) g[k] = (float)(t[k] / s);
  if (cudaMemcpyToSymbol(c_gauss, g, sizeof(g)) != cudaSuccess) return 1;
  g_gauss_set[device] = true;
  return 0;
}

size_t image_loss_temp_bytes(int W, int H) { return 256 + (size_t)9 * W * H * sizeof(float); }

void launch_image_loss(const float4* img, const float4* tgt, int W, int H, float lam, float* loss, float4* grad,
                       void* temp, cudaStream_t st) {
  double* acc = reinterpret_cast<double*>(temp);
  float* part = reinterpret_cast<float*>(reinterpret_cast<char*>(temp) + 256);
  const double n3 = 3.0 * (double)W * (double)H;
  cudaMemsetAsync(acc, 0, 2 * sizeof(double), st);
  dim3 grid((W + SS_TO - 1) / SS_TO, (H + SS_TO - 1) / SS_TO, 3), block(SS_THREADS);
  k_ssim_fwd<<<grid, block, 0, st>>>(img, tgt, W, H, (float)(-lam / n3), part, acc);
  k_ssim_bwd<<<grid, block, 0, st>>>(img, tgt, W, H, part, (float)((1.0 - lam) / n3), grad);
  k_loss_finish<<<1, 1, 0, st>>>(acc, n3, lam, loss);
  note_launches(3);
}

}  // namespace ts
