// Per-splat preprocess (forward) and its adjoint.
//
// Forward, one thread per (view, splat) item:
//   * culling, tile rect and depth key in the FP32 binning specification:
//     single correctly rounded operations in a fixed order (__fmul_rn,
//     __fadd_rn, __fdiv_rn, __fsqrt_rn), so the tile/depth key list is
//     bit-identical to the specification it implements;
//   * the raster record: homography rows of the closed-form ray-splat
//     intersection (Sec. 3.1) in centred pixel coordinates, the opacity and
//     the camera-facing tangent frame for normal mapping (Eq. 7).
// Backward, one thread per item: chains the per-item record gradients
// accumulated by the rasteriser back to means, quaternions, scales and
// opacities.
#include "kernels.h"
#include "prof.h"

namespace ts {

// Rotation columns (t_u, t_v, n) of the normalised quaternion, spec order.
__device__ __forceinline__ void rot_cols_spec(float4 q, float tu[3], float tv[3], float n[3]) {
  float w = q.x, x = q.y, y = q.z, z = q.w;
  float nrm = __fsqrt_rn(__fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(w, w), __fmul_rn(x, x)), __fmul_rn(y, y)),
                                   __fmul_rn(z, z)));
  w = __fdiv_rn(w, nrm);
  x = __fdiv_rn(x, nrm);
  y = __fdiv_rn(y, nrm);
  z = __fdiv_rn(z, nrm);
  float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
  float xy = __fmul_rn(x, y), xz = __fmul_rn(x, z), yz = __fmul_rn(y, z);
  float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, z);
  tu[0] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(yy, zz)));
  tu[1] = __fmul_rn(2.f, __fadd_rn(xy, wz));
  tu[2] = __fmul_rn(2.f, __fsub_rn(xz, wy));
  tv[0] = __fmul_rn(2.f, __fsub_rn(xy, wz));
  tv[1] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(xx, zz)));
  tv[2] = __fmul_rn(2.f, __fadd_rn(yz, wx));
  n[0] = __fmul_rn(2.f, __fadd_rn(xz, wy));
  n[1] = __fmul_rn(2.f, __fsub_rn(yz, wx));
  n[2] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(xx, yy)));
}

__device__ __forceinline__ float cam_row_spec(const float* R, int r, float t, float c0, float c1, float c2) {
  return __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(R[3 * r], c0), __fmul_rn(R[3 * r + 1], c1)),
                             __fmul_rn(R[3 * r + 2], c2)),
                   t);
}

__global__ void __launch_bounds__(256) k_preprocess(ViewTable vt, Record* __restrict__ rec,
                                                     uint32_t* __restrict__ counts,
                                                     uint64_t* __restrict__ depth_keys,
                                                     uint32_t* __restrict__ item_ids, int4* __restrict__ rects) {
  const int item = blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= vt.n_items) return;
  const int v = find_view_item(vt, item);
  const ViewDesc& V = vt.v[v];
  const int k = item - V.item_off;
  item_ids[item] = (uint32_t)item;
  counts[item] = 0;
  depth_keys[item] = ~0ull;
  if (k >= V.n_splats) return;

  const float4 p4 = V.means[k];
  const float4 q = V.quats[k];
  const float2 s = V.scales[k];
  const float o = V.opacity[k];
  const float p[3] = {p4.x, p4.y, p4.z};
  float tu[3], tv[3], n[3];
  rot_cols_spec(q, tu, tv, n);

  // 3-sigma support corners (Sec. 3.3, S_sigma = 3) and their projection
  const float eu = __fmul_rn(3.f, s.x), ev = __fmul_rn(3.f, s.y);
  float du[3], dv[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    du[i] = __fmul_rn(eu, tu[i]);
    dv[i] = __fmul_rn(ev, tv[i]);
  }
  bool front = true;
  float xmin = 0.f, xmax = 0.f, ymin = 0.f, ymax = 0.f;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const bool pa = (c & 1), pb = (c & 2);
    float cw[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      float a = pa ? __fadd_rn(p[i], du[i]) : __fsub_rn(p[i], du[i]);
      cw[i] = pb ? __fadd_rn(a, dv[i]) : __fsub_rn(a, dv[i]);
    }
    const float X = cam_row_spec(V.R, 0, V.t[0], cw[0], cw[1], cw[2]);
    const float Y = cam_row_spec(V.R, 1, V.t[1], cw[0], cw[1], cw[2]);
    const float Z = cam_row_spec(V.R, 2, V.t[2], cw[0], cw[1], cw[2]);
    front = front && (Z > kNear());
    const float px = __fadd_rn(__fmul_rn(V.fx, __fdiv_rn(X, Z)), V.cx);
    const float py = __fadd_rn(__fmul_rn(V.fy, __fdiv_rn(Y, Z)), V.cy);
    if (c == 0) {
      xmin = xmax = px;
      ymin = ymax = py;
    } else {
      xmin = fminf(xmin, px);
      xmax = fmaxf(xmax, px);
      ymin = fminf(ymin, py);
      ymax = fmaxf(ymax, py);
    }
  }
  if (!front) return;
  const float tx0 = fmaxf(0.f, floorf(__fmul_rn(xmin, 0.0625f)));
  const float tx1 = fminf((float)(V.tiles_x - 1), floorf(__fmul_rn(xmax, 0.0625f)));
  const float ty0 = fmaxf(0.f, floorf(__fmul_rn(ymin, 0.0625f)));
  const float ty1 = fminf((float)(V.tiles_y - 1), floorf(__fmul_rn(ymax, 0.0625f)));
  if (!(tx0 <= tx1 && ty0 <= ty1)) return;
  if (!(o >= kAlphaMin())) return;
  const float depth = cam_row_spec(V.R, 2, V.t[2], p[0], p[1], p[2]);
  if (!(depth > kNear())) return;

  const int ix0 = (int)tx0, ix1 = (int)tx1, iy0 = (int)ty0, iy1 = (int)ty1;
  counts[item] = (uint32_t)((ix1 - ix0 + 1) * (iy1 - iy0 + 1));
  rects[item] = make_int4(ix0, ix1, iy0, iy1);
  depth_keys[item] = ((uint64_t)v << 32) | (uint64_t)__float_as_uint(depth);

  // ---- raster record (regular FP32, not part of the key specification) ----
  const float* R = V.R;
  float pc[3], tuc[3], tvc[3], nc[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    pc[r] = R[3 * r] * p[0] + R[3 * r + 1] * p[1] + R[3 * r + 2] * p[2] + V.t[r];
    tuc[r] = R[3 * r] * tu[0] + R[3 * r + 1] * tu[1] + R[3 * r + 2] * tu[2];
    tvc[r] = R[3 * r] * tv[0] + R[3 * r + 1] * tv[1] + R[3 * r + 2] * tv[2];
    nc[r] = R[3 * r] * n[0] + R[3 * r + 1] * n[1] + R[3 * r + 2] * n[2];
  }
  const float D = pc[0] * nc[0] + pc[1] * nc[1] + pc[2] * nc[2];
  const float Pu = pc[0] * tuc[0] + pc[1] * tuc[1] + pc[2] * tuc[2];
  const float Pv = pc[0] * tvc[0] + pc[1] * tvc[1] + pc[2] * tvc[2];
  const float isu = 1.f / s.x, isv = 1.f / s.y;
  float hu[3], hv[3], hw[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    hu[i] = (D * tuc[i] - Pu * nc[i]) * isu;
    hv[i] = (D * tvc[i] - Pv * nc[i]) * isv;
    hw[i] = nc[i];
  }
  // d-space rows -> centred pixel rows: d = (x'/fx, y'/fy, 1)
  const float ifx = 1.f / V.fx, ify = 1.f / V.fy;
  hu[0] *= ifx; hu[1] *= ify;
  hv[0] *= ifx; hv[1] *= ify;
  hw[0] *= ifx; hw[1] *= ify;
  // normal turned to face the camera: (p - o).n = p_c . n_c > 0 -> flip
  const float sg = (D > 0.f) ? -1.f : 1.f;
  Record r;
  r.r0 = make_float4(hu[0], hv[0], hu[1], hv[1]);
  r.r1 = make_float4(hu[2], hv[2], hw[0], hw[1]);
  r.r2 = make_float4(hw[2], o, tu[0], tu[1]);
  r.r3 = make_float4(tu[2], tv[0], tv[1], tv[2]);
  r.r4 = make_float4(sg * n[0], sg * n[1], sg * n[2], D);  // D: hit depth = D / den
  rec[item] = r;
}

void launch_preprocess(const ViewTable& vt, Record* rec, uint32_t* counts, uint64_t* depth_keys,
                       uint32_t* item_ids, int4* rects, cudaStream_t st) {
  if (vt.n_items == 0) return;
  k_preprocess<<<(vt.n_items + 255) / 256, 256, 0, st>>>(vt, rec, counts, depth_keys, item_ids, rects);
  note_launches(1);
}

// ---------------------------------------------------------------------------
// Adjoint.  g_items[item][14]: 0-2 d/dh_u, 3-5 d/dh_v, 6-8 d/dh_w (centred
// pixel rows), 9 d/do, 10-12 the torque tau of the normal-mapping frame
// (world): a rotation by a small angle vector w changes the loss by tau . w,
// 13 d/dD (D = p_c . n_c, the plane offset of the depth channel).
// The per-splat sums arrive in float64 (accumulated across warps without
// FP32 cancellation); the chain itself runs in float32 (a float64 chain was
// measured: no accuracy change, 10x the time on this part).
__global__ void __launch_bounds__(256) k_preprocess_bwd(ViewTable vt, const double* __restrict__ g_items,
                                                         GradTable g) {
  using R_t = float;
  const int item = blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= vt.n_items) return;
  const int v = find_view_item(vt, item);
  const ViewDesc& V = vt.v[v];
  const int k = item - V.item_off;
  if (k >= V.n_splats) return;
  const double2* gp2 = reinterpret_cast<const double2*>(g_items + (size_t)item * kRecGradStride);
  R_t gi[kRecGradStride];
#pragma unroll
  for (int i = 0; i < kRecGradStride / 2; ++i) {
    const double2 a = gp2[i];
    gi[2 * i] = a.x;
    gi[2 * i + 1] = a.y;
  }
  bool any = false;
#pragma unroll
  for (int i = 0; i < kRecGrads; ++i) any |= (gi[i] != 0.0);
  if (!any) return;

  const float4 p4 = V.means[k];
  const float4 q = V.quats[k];
  const float2 s = V.scales[k];
  const R_t p[3] = {p4.x, p4.y, p4.z};
  const R_t qn = sqrt((R_t)q.x * q.x + (R_t)q.y * q.y + (R_t)q.z * q.z + (R_t)q.w * q.w);
  const R_t iq = R_t(1) / qn;
  const R_t w = q.x * iq, x = q.y * iq, y = q.z * iq, z = q.w * iq;
  const R_t tu[3] = {1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)};
  const R_t tv[3] = {2 * (x * y - w * z), 1 - 2 * (x * x + z * z), 2 * (y * z + w * x)};
  const R_t n[3] = {2 * (x * z + w * y), 2 * (y * z - w * x), 1 - 2 * (x * x + y * y)};
  R_t Rm[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) Rm[i] = V.R[i];
  R_t pc[3], tuc[3], tvc[3], nc[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    pc[r] = Rm[3 * r] * p[0] + Rm[3 * r + 1] * p[1] + Rm[3 * r + 2] * p[2] + (R_t)V.t[r];
    tuc[r] = Rm[3 * r] * tu[0] + Rm[3 * r + 1] * tu[1] + Rm[3 * r + 2] * tu[2];
    tvc[r] = Rm[3 * r] * tv[0] + Rm[3 * r + 1] * tv[1] + Rm[3 * r + 2] * tv[2];
    nc[r] = Rm[3 * r] * n[0] + Rm[3 * r + 1] * n[1] + Rm[3 * r + 2] * n[2];
  }
  const R_t D = pc[0] * nc[0] + pc[1] * nc[1] + pc[2] * nc[2];
  const R_t Pu = pc[0] * tuc[0] + pc[1] * tuc[1] + pc[2] * tuc[2];
  const R_t Pv = pc[0] * tvc[0] + pc[1] * tvc[1] + pc[2] * tvc[2];
  const R_t isu = R_t(1) / (R_t)s.x, isv = R_t(1) / (R_t)s.y;
  const R_t ifx = R_t(1) / (R_t)V.fx, ify = R_t(1) / (R_t)V.fy;
  // centred pixel rows -> d-space rows
  const R_t ghu[3] = {gi[0] * ifx, gi[1] * ify, gi[2]};
  const R_t ghv[3] = {gi[3] * ifx, gi[4] * ify, gi[5]};
  const R_t ghw[3] = {gi[6] * ifx, gi[7] * ify, gi[8]};
  R_t gpc[3] = {0, 0, 0}, gtuc[3] = {0, 0, 0}, gtvc[3] = {0, 0, 0};
  R_t gnc[3] = {ghw[0], ghw[1], ghw[2]};
  // h_u = (D t_u - P_u n)/s_u, h_v likewise, h_w = n
  R_t gD = gi[13], gPu = 0, gPv = 0, gsu = 0, gsv = 0;  // gi[13]: D through the depth channel
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const R_t hu = (D * tuc[i] - Pu * nc[i]) * isu;
    const R_t hv = (D * tvc[i] - Pv * nc[i]) * isv;
    gD += (ghu[i] * tuc[i]) * isu + (ghv[i] * tvc[i]) * isv;
    gtuc[i] += D * ghu[i] * isu;
    gtvc[i] += D * ghv[i] * isv;
    gPu -= ghu[i] * nc[i] * isu;
    gPv -= ghv[i] * nc[i] * isv;
    gnc[i] -= Pu * ghu[i] * isu + Pv * ghv[i] * isv;
    gsu -= ghu[i] * hu * isu;
    gsv -= ghv[i] * hv * isv;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    gpc[i] += gD * nc[i] + gPu * tuc[i] + gPv * tvc[i];
    gnc[i] += gD * pc[i];
    gtuc[i] += gPu * pc[i];
    gtvc[i] += gPv * pc[i];
  }
  // camera -> world (R^T), plus the normal-mapping frame: column gradients
  // g_f = (tau x f) / 2 for the orthonormal columns f = t_u, t_v, n give
  // sum_f f x g_f = tau, the same rotation gradient as the full 3x3 frame
  // gradient (the camera-facing flip of n cancels: n_f = -n, g_n = -g_nf)
  const R_t ta[3] = {gi[10], gi[11], gi[12]};
  const R_t htu[3] = {R_t(0.5) * (ta[1] * tu[2] - ta[2] * tu[1]), R_t(0.5) * (ta[2] * tu[0] - ta[0] * tu[2]),
                      R_t(0.5) * (ta[0] * tu[1] - ta[1] * tu[0])};
  const R_t htv[3] = {R_t(0.5) * (ta[1] * tv[2] - ta[2] * tv[1]), R_t(0.5) * (ta[2] * tv[0] - ta[0] * tv[2]),
                      R_t(0.5) * (ta[0] * tv[1] - ta[1] * tv[0])};
  const R_t hn[3] = {R_t(0.5) * (ta[1] * n[2] - ta[2] * n[1]), R_t(0.5) * (ta[2] * n[0] - ta[0] * n[2]),
                     R_t(0.5) * (ta[0] * n[1] - ta[1] * n[0])};
  R_t gpw[3], gtu[3], gtv[3], gn[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    gpw[i] = Rm[i] * gpc[0] + Rm[3 + i] * gpc[1] + Rm[6 + i] * gpc[2];
    gtu[i] = Rm[i] * gtuc[0] + Rm[3 + i] * gtuc[1] + Rm[6 + i] * gtuc[2] + htu[i];
    gtv[i] = Rm[i] * gtvc[0] + Rm[3 + i] * gtvc[1] + Rm[6 + i] * gtvc[2] + htv[i];
    gn[i] = Rm[i] * gnc[0] + Rm[3 + i] * gnc[1] + Rm[6 + i] * gnc[2] + hn[i];
  }
  // rotation matrix of the unit quaternion -> quaternion
  const R_t gw = 2 * (z * gtu[1] - y * gtu[2] - z * gtv[0] + x * gtv[2] + y * gn[0] - x * gn[1]);
  const R_t gx = 2 * (y * gtu[1] + z * gtu[2] + y * gtv[0] - 2 * x * gtv[1] + w * gtv[2] + z * gn[0] - w * gn[1] -
                      2 * x * gn[2]);
  const R_t gy = 2 * (-2 * y * gtu[0] + x * gtu[1] - w * gtu[2] + x * gtv[0] + z * gtv[2] + w * gn[0] + z * gn[1] -
                      2 * y * gn[2]);
  const R_t gz = 2 * (-2 * z * gtu[0] + w * gtu[1] + x * gtu[2] - w * gtv[0] - 2 * z * gtv[1] + y * gtv[2] +
                      x * gn[0] + y * gn[1]);
  const R_t dp = w * gw + x * gx + y * gy + z * gz;
  if (g.quats) {
    float* gq = g.quats + (size_t)k * 4;
    red_add_v4(gq, (float)((gw - w * dp) * iq), (float)((gx - x * dp) * iq), (float)((gy - y * dp) * iq),
               (float)((gz - z * dp) * iq));
  }
  if (g.means) {
    float* gm = g.means + (size_t)k * 3;
    red_add(gm, (float)gpw[0]);
    red_add(gm + 1, (float)gpw[1]);
    red_add(gm + 2, (float)gpw[2]);
  }
  if (g.scales) {
    red_add(g.scales + (size_t)k * 2, (float)gsu);
    red_add(g.scales + (size_t)k * 2 + 1, (float)gsv);
  }
  if (g.opacity) red_add(g.opacity + k, (float)gi[9]);
}

void launch_preprocess_bwd(const ViewTable& vt, const double* g_items, const GradTable& g, cudaStream_t st) {
  if (vt.n_items == 0) return;
  k_preprocess_bwd<<<(vt.n_items + 255) / 256, 256, 0, st>>>(vt, g_items, g);
  note_launches(1);
}

}  // namespace ts
