// Normal-consistency loss of Sec. 3.6, L_n = 1 - N~^T N, on a saved view.
//
// From the forward's blended depth Zs, coverage A and G-buffer normal N:
//   D = Zs / A (expected camera depth) where A >= 0.5, back-projected to
//   P = D (x'/fx, y'/fy, 1); N~ = normalize((P[y+1] - P[y-1]) x (P[x+1] - P[x-1]))
//   (camera space, facing the camera), turned to world space by R^T; N^ =
//   N / |N|.  Interior pixels whose own and four neighbours' coverage is
//   >= 0.5 (and whose normal and cross product are non-zero) add
//   1 - N~ . N^; L_n = weight x sum / ((W - 2)(H - 2)).
// Two passes: k_normal_loss computes each counted pixel's term, its
// gradient w.r.t. its own normal channel and its four depth derivatives
// (one per neighbour it reads); k_normal_gather collects, per pixel, the
// derivatives its neighbours sent it and turns dL/dD into dL/dZs and dL/dA.
// Deterministic: no atomics except one float64 add per CTA for the sum.
#include "kernels.h"
#include "prof.h"

namespace ts {

namespace {

constexpr float kCoverMin = 0.5f;
constexpr int NL_THREADS = 256;

__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

struct NLView {
  int W, H;
  float fx, fy, cx, cy;
  float R[9];
  const float4* gbuf;  // [H][W][2]
  const float* acc;
  const float* zsum;
  float4* gN;   // out: dL/dN (xyz) of the pixel's own term
  float4* gDn;  // out: dL/dD sent to (x+1, x-1, y+1, y-1)
  float4* gnorm;  // out: dL/dN (xyz), dL/dA (w)
  float* gzsum;   // out: dL/dZs
};

__device__ __forceinline__ float depth_at(const NLView& v, int x, int y, bool& ok) {
  const int p = y * v.W + x;
  const float a = v.acc[p];
  ok = a >= kCoverMin;
  return ok ? v.zsum[p] / a : 0.f;
}

__device__ __forceinline__ float3 ray_at(const NLView& v, int x, int y) {
  return make_float3(((float)x + 0.5f - v.cx) / v.fx, ((float)y + 0.5f - v.cy) / v.fy, 1.f);
}

__global__ void __launch_bounds__(NL_THREADS) k_normal_loss(NLView v, float scale, double* __restrict__ sum) {
  __shared__ double red[NL_THREADS / 32];
  const long long np = (long long)v.W * v.H;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float term = 0.f;
  if (p < np) {
    const int x = (int)(p % v.W), y = (int)(p / v.W);
    float4 gN = make_float4(0.f, 0.f, 0.f, 0.f), gD = make_float4(0.f, 0.f, 0.f, 0.f);
    if (x >= 1 && y >= 1 && x < v.W - 1 && y < v.H - 1) {
      bool o0, o1, o2, o3, o4;
      depth_at(v, x, y, o0);
      const float dxp = depth_at(v, x + 1, y, o1), dxm = depth_at(v, x - 1, y, o2);
      const float dyp = depth_at(v, x, y + 1, o3), dym = depth_at(v, x, y - 1, o4);
      const float4 g1 = v.gbuf[2 * p + 1];
      const float3 N = make_float3(g1.y, g1.z, g1.w);  // channels 5-7
      const float nl = sqrtf(dot3(N, N));
      const float3 rxp = ray_at(v, x + 1, y), rxm = ray_at(v, x - 1, y);
      const float3 ryp = ray_at(v, x, y + 1), rym = ray_at(v, x, y - 1);
      const float3 Pxp = make_float3(dxp * rxp.x, dxp * rxp.y, dxp), Pxm = make_float3(dxm * rxm.x, dxm * rxm.y, dxm);
      const float3 Pyp = make_float3(dyp * ryp.x, dyp * ryp.y, dyp), Pym = make_float3(dym * rym.x, dym * rym.y, dym);
      const float3 ex = sub3(Pxp, Pxm), ey = sub3(Pyp, Pym);
      const float3 c = cross3(ey, ex);
      const float cl = sqrtf(dot3(c, c));
      if (o0 && o1 && o2 && o3 && o4 && nl >= 1e-12f && cl > 0.f) {
        const float ic = 1.f / cl, in = 1.f / nl;
        const float3 Nt = make_float3(c.x * ic, c.y * ic, c.z * ic);  // camera space
        const float* R = v.R;
        // rendered normal in camera space: m = R N^
        const float3 Nh = make_float3(N.x * in, N.y * in, N.z * in);
        const float3 m = make_float3(R[0] * Nh.x + R[1] * Nh.y + R[2] * Nh.z, R[3] * Nh.x + R[4] * Nh.y + R[5] * Nh.z,
                                     R[6] * Nh.x + R[7] * Nh.y + R[8] * Nh.z);
        const float d = dot3(Nt, m);
        term = 1.f - d;
        // dl/dm = -Nt -> dl/dN^ = -R^T Nt -> through the normalisation
        const float3 gNh = make_float3(-(R[0] * Nt.x + R[3] * Nt.y + R[6] * Nt.z),
                                       -(R[1] * Nt.x + R[4] * Nt.y + R[7] * Nt.z),
                                       -(R[2] * Nt.x + R[5] * Nt.y + R[8] * Nt.z));
        const float pr = dot3(Nh, gNh);
        gN = make_float4(scale * (gNh.x - Nh.x * pr) * in, scale * (gNh.y - Nh.y * pr) * in,
                         scale * (gNh.z - Nh.z * pr) * in, 0.f);
        // dl/dc = -(m - Nt (Nt . m)) / |c|; c = ey x ex
        const float3 gc = make_float3(-(m.x - Nt.x * d) * ic, -(m.y - Nt.y * d) * ic, -(m.z - Nt.z * d) * ic);
        const float3 gex = cross3(gc, ey);  // d(gc . (ey x ex)) / d ex
        const float3 gey = cross3(ex, gc);  // d(gc . (ey x ex)) / d ey
        // P = D r: dl/dD = dl/dP . r; ex = P(x+1) - P(x-1), ey = P(y+1) - P(y-1)
        gD = make_float4(scale * dot3(gex, rxp), -scale * dot3(gex, rxm), scale * dot3(gey, ryp),
                         -scale * dot3(gey, rym));
      }
    }
    v.gN[p] = gN;
    v.gDn[p] = gD;
  }
  double t = term;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NL_THREADS / 32; ++w) s += red[w];
    if (s != 0.0) atomicAdd(sum, s);
  }
}

__global__ void __launch_bounds__(NL_THREADS) k_normal_gather(NLView v) {
  const long long np = (long long)v.W * v.H;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int x = (int)(p % v.W), y = (int)(p / v.W);
  // dL/dD(x, y): what the neighbours that read this pixel's depth sent it
  float gD = 0.f;
  if (x >= 1) gD += v.gDn[p - 1].x;         // (x-1, y) reads it as its x+1
  if (x + 1 < v.W) gD += v.gDn[p + 1].y;    // (x+1, y) reads it as its x-1
  if (y >= 1) gD += v.gDn[p - v.W].z;       // (x, y-1) reads it as its y+1
  if (y + 1 < v.H) gD += v.gDn[p + v.W].w;  // (x, y+1) reads it as its y-1
  const float4 gN = v.gN[p];
  float gA = 0.f, gZ = 0.f;
  const float a = v.acc[p];
  if (gD != 0.f && a >= kCoverMin) {  // D = Zs / A
    gZ = gD / a;
    gA = -gD * v.zsum[p] / (a * a);
  }
  v.gnorm[p] = make_float4(gN.x, gN.y, gN.z, gA);
  v.gzsum[p] = gZ;
}

__global__ void k_normal_finish(const double* __restrict__ sum, double denom, float weight, float* __restrict__ loss) {
  loss[0] = (float)(weight * sum[0] / denom);
}

}  // namespace

size_t normal_loss_temp_bytes(int W, int H) { return 256 + (size_t)W * H * 2 * sizeof(float4); }

void launch_normal_loss(const ViewDesc& V, float weight, float* loss, float4* gnorm, float* gzsum, void* temp,
                        cudaStream_t st) {
  NLView v;
  v.W = V.W;
  v.H = V.H;
  v.fx = V.fx;
  v.fy = V.fy;
  v.cx = V.cx;
  v.cy = V.cy;
  for (int i = 0; i < 9; ++i) v.R[i] = V.R[i];
  v.gbuf = V.gbuf;
  v.acc = V.acc;
  v.zsum = V.zsum;
  double* sum = reinterpret_cast<double*>(temp);
  const long long np = (long long)V.W * V.H;
  v.gN = reinterpret_cast<float4*>(reinterpret_cast<char*>(temp) + 256);
  v.gDn = v.gN + np;
  v.gnorm = gnorm;
  v.gzsum = gzsum;
  const double denom = (V.W > 2 && V.H > 2) ? (double)(V.W - 2) * (double)(V.H - 2) : 1.0;
  const float scale = (float)(weight / denom);
  cudaMemsetAsync(sum, 0, sizeof(double), st);
  const unsigned blocks = (unsigned)((np + NL_THREADS - 1) / NL_THREADS);
  k_normal_loss<<<blocks, NL_THREADS, 0, st>>>(v, scale, sum);
  k_normal_gather<<<blocks, NL_THREADS, 0, st>>>(v);
  k_normal_finish<<<1, 1, 0, st>>>(sum, denom, weight, loss);
  note_launches(3);
}

}  // namespace ts
