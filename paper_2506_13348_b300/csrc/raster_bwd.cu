// Backward rasteriser: one thread per pixel, one warp per 8x4 pixel block,
// two CTAs of 4 warps per 16x16 tile (as the forward).
//
// Input: dL/dX (the 8 G-buffer channels) and dL/dA per pixel, written by the
// shading adjoint (Eq. 10-12, k_shade_bwd), plus the forward's saved
// transmittance and last blended index per pixel.
// Main loop: each warp (an 8x4 pixel block) walks the tile's list back to
// front on its own, from the last fragment any of its pixels blended, with
// no block-wide barrier.  Each fragment's (u,v), alpha and texel value are
// recomputed from the splat's record (the per-pixel fragment lists are never
// stored); the transmittance in front of it is recovered by division
// (alpha <= 0.99) and the colour behind it by the usual recurrence.
// Reductions (all lanes of a warp work on the same splat at a time):
//   * the 14 record gradients of the fragment are summed over the warp by a
//     halving reduce-scatter (16 shuffles), after which one lane per value
//     adds it once per warp;
//   * texel gradients are summed per bilinear cell over the warp (a
//     reduce-scatter through shuffles) before one reduction per cell; lanes
//     whose cell few others share add their own values directly.
#include "raster.cuh"
#include "shading.cuh"
#include "kernels.h"
#include "prof.h"

namespace ts {

template <int DT, int FEAT>
__global__ void __launch_bounds__(32 * kRasterWarps, ((FEAT & FEAT_IND) ? 2 : 3) * kCtasPerTile) k_raster_bwd(ViewTable vt, const Record* __restrict__ rec,
                                                                  const uint32_t* __restrict__ pair_items,
                                                                  const uint2* __restrict__ ranges,
                                                                  const float4* __restrict__ gxa,
                                                                  double* __restrict__ g_items, GradTable g) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr bool IND = (FEAT & FEAT_IND) != 0, N2 = (FEAT & FEAT_N2) != 0;
  // indirect light: per lane dL/dl (3) and the SH basis (9), value-major
  __shared__ __align__(16) float s_sh[IND ? kRasterWarps : 1][12][36];
  __shared__ __align__(16) float4 s_rec[kRasterWarps][2][32][3];  // the records of this chunk and the next
  __shared__ uint32_t s_item[kRasterWarps][2][32];
  const int warp = threadIdx.x >> 5;
  const int tile = raster_tile(vt);
  if ((unsigned)tile >= (unsigned)vt.n_tiles) return;  // an order from a failed sort (flag set)
  if (lists_failed(vt)) return;                        // the forward marked the image invalid
  const int v = find_view(vt, tile);
  const ViewDesc& V = vt.v[v];
  int px, py;
  pixel_of(tile - V.tile_off, V.tiles_x, raster_block(), px, py);
  const bool inside = px < V.W && py < V.H;
  const float xp = (float)px + 0.5f - V.cx;
  const float yp = (float)py + 0.5f - V.cy;
  const int lo = (int)ranges[tile].x;
  const int T = V.T;
  const float Ts6 = (float)T * (1.0f / 6.0f);
  const int lane = threadIdx.x & 31;

  float gX[8], gA = 0.f, gZ = 0.f, Tcur = 1.f;
  float gXi[3] = {0.f, 0.f, 0.f};  // dL/dX_ind (indirect light channel)
  float3 wo = make_float3(0.f, 0.f, 1.f);
  const int shK = (V.sh_deg + 1) * (V.sh_deg + 1);
  int last = -1;
#pragma unroll
  for (int c = 0; c < 8; ++c) gX[c] = 0.f;
  if (inside) {
    const int pix = py * V.W + px;
    const long long gp = (long long)V.pix_off + pix;
    const float4 a = gxa[3 * gp], b = gxa[3 * gp + 1];
    gX[0] = a.x; gX[1] = a.y; gX[2] = a.z; gX[3] = a.w;
    gX[4] = b.x; gX[5] = b.y; gX[6] = b.z; gX[7] = b.w;
    const float4 c = gxa[3 * gp + 2];
    gA = c.x;
    gZ = c.y;  // dL/d(blended depth), zero unless a depth loss is in use
    Tcur = V.trans[pix];
    last = V.last[pix];
    if (IND) {
      const float4 q = V.gxind[pix];
      gXi[0] = q.x;
      gXi[1] = q.y;
      gXi[2] = q.z;
      const float3 d = world_ray(V, xp, yp);
      const float id = rsqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
      wo = make_float3(-d.x * id, -d.y * id, -d.z * id);
    }
  }
  const int hi = __reduce_max_sync(FULL, last);

  // dL/dX . (colour behind the current fragment) + dL/dA . (coverage behind it)
  float P = 0.f;

  // the warp's 8x4 pixel block in centred pixel coordinates (for culling)
  const float bx0 = (float)(px - (lane & 7)) + 0.5f - V.cx, bx1 = bx0 + 7.f;
  const float by0 = (float)(py - (lane >> 3)) + 0.5f - V.cy, by1 = by0 + 3.f;

  // The list is taken 32 entries at a time, back to front: lane t's entry
  // ch - t has the first 48 bytes of its record (the rows the block test and
  // the fragment need; the rest is read when an entry is processed) copied
  // into shared memory by cp.async one chunk ahead (the next chunk's copy runs while the warp works on this one; the
  // item ids run one chunk further ahead in a register); the lane tests it
  // against the warp's block and only the surviving entries are processed,
  // in back-to-front order.
  auto issue = [&](int b, int c, uint32_t it) {
    if (c - lane >= lo) {
      const float4* rp = reinterpret_cast<const float4*>(rec + it);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(&s_rec[warp][b][lane][q]);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(rp + q) : "memory");
      }
      s_item[warp][b][lane] = it;
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  uint32_t it_next = (hi - lane >= lo) ? __ldg(pair_items + hi - lane) : 0u;
  issue(0, hi, it_next);
  it_next = (hi - 32 - lane >= lo) ? __ldg(pair_items + hi - 32 - lane) : 0u;
  int buf = 0;
  for (int ch = hi; ch >= lo; ch -= 32, buf ^= 1) {
    issue(buf ^ 1, ch - 32, it_next);
    it_next = (ch - 64 - lane >= lo) ? __ldg(pair_items + ch - 64 - lane) : 0u;
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncwarp();
    const int e = ch - lane;
    bool cand = false;
    if (e >= lo) {
      Record c;
      c.r0 = s_rec[warp][buf][lane][0];
      c.r1 = s_rec[warp][buf][lane][1];
      c.r2 = s_rec[warp][buf][lane][2];
      cand = block_may_hit(c, bx0, bx1, by0, by1);
    }
    const unsigned cmask = __ballot_sync(FULL, cand);
  for (unsigned cm = cmask; cm; cm &= cm - 1) {
    const int t = __ffs(cm) - 1;
    const int j = ch - t;
    const uint32_t item = s_item[warp][buf][t];
    Record r;
    r.r0 = s_rec[warp][buf][t][0];
    r.r1 = s_rec[warp][buf][t][1];
    r.r2 = s_rec[warp][buf][t][2];
    Frag f;
    const bool ok = (j <= last) && eval_frag(r, xp, yp, f);
    if (__any_sync(FULL, ok)) {
      {
        const float4* rp = reinterpret_cast<const float4*>(rec + item);
        r.r3 = __ldg(rp + 3);
        r.r4 = __ldg(rp + 4);
      }
      const long long splat = (long long)item - V.item_off;
      float t8[8], w4[4] = {0.f, 0.f, 0.f, 0.f};
      TexSample ts_;
      ts_.ia = ts_.ib = ts_.ja = ts_.jb = 0;
      float gi[kRecGrads];
      float shv[12];  // indirect light: dL/dl (3), basis Y (9)
#pragma unroll
      for (int q = 0; q < 12; ++q) shv[q] = 0.f;
      if (ok) {
        ts_ = tex_setup(f.u, f.v, T);
        const float om = 1.f - f.alpha;
        // transmittance in front of the fragment: om >= 0.01, and the
        // approximate quotient (2 ulp) keeps the recovered T within a few
        // 1e-6 relative over the ~100 fragments of a pixel
        const float Tb = __fdividef(Tcur, om);
        const float wgt = f.alpha * Tb;
        // g8: dL/dX pulled back to the texture channels (0-4 direct, 5-7
        // through the normal map n = [t_u t_v n_f] n^t, i.e. R'^T dL/dN)
        float g8[8];
#pragma unroll
        for (int c = 0; c < 5; ++c) g8[c] = gX[c];
        // e = dL/dn^t (tangent normal); with two stored components n^t is
        // not linear in the texels: the corner loop takes channels 0-4 only
        // and the normal's share is added once n^t is known
        const float e0 = r.r2.z * gX[5] + r.r2.w * gX[6] + r.r3.x * gX[7];
        const float e1 = r.r3.y * gX[5] + r.r3.z * gX[6] + r.r3.w * gX[7];
        const float e2 = r.r4.x * gX[5] + r.r4.y * gX[6] + r.r4.z * gX[7];
        g8[5] = N2 ? 0.f : e0;
        g8[6] = N2 ? 0.f : e1;
        g8[7] = N2 ? 0.f : e2;
        // stream the four bilinear corners: only the projections g8 . texel
        // and the tangent normal are needed
        const float hx = 1.f - ts_.fx, hy = 1.f - ts_.fy;
        w4[0] = hx * hy; w4[1] = ts_.fx * hy; w4[2] = hx * ts_.fy; w4[3] = ts_.fx * ts_.fy;
        float2 nt01 = f2(0.f, 0.f), dxy = f2(0.f, 0.f);
        float nt2 = 0.f, gxx = 0.f;
        // indirect light, two-component normals: d(interpolated normal
        // channels)/d(texel-space u, v)
        float dnu[3] = {0.f, 0.f, 0.f}, dnv[3] = {0.f, 0.f, 0.f};
        const float2 g01 = f2(g8[0], g8[1]), g23 = f2(g8[2], g8[3]), g45 = f2(g8[4], g8[5]), g67 = f2(g8[6], g8[7]);
        // (two 16-byte loads per float32 texel: one 32-byte load holds eight
        // more registers live and spills here)
        const long long base = splat * (long long)T * T;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int jj = (k & 2) ? ts_.jb : ts_.ja;
          const int ii = (k & 1) ? ts_.ib : ts_.ia;
          float cv[8];
          load_texel(V.texels, DT, base + jj * T + ii, cv);
          float2 acc = mul2(g01, f2(cv[0], cv[1]));
          acc = fma2(g23, f2(cv[2], cv[3]), acc);
          acc = fma2(g45, f2(cv[4], cv[5]), acc);
          acc = fma2(g67, f2(cv[6], cv[7]), acc);
          const float tdot = acc.x + acc.y;
          nt01 = fma2(f2(w4[k], w4[k]), f2(cv[5], cv[6]), nt01);
          nt2 = fmaf(w4[k], cv[7], nt2);
          gxx = fmaf(w4[k], tdot, gxx);
          const float wyk = (k & 2) ? ts_.fy : hy;
          const float wxk = (k & 1) ? ts_.fx : hx;
          dxy = fma2(f2((k & 1) ? wyk : -wyk, (k & 2) ? wxk : -wxk), f2(tdot, tdot), dxy);
          if (IND || N2) {
            const float au = (k & 1) ? wyk : -wyk, av = (k & 2) ? wxk : -wxk;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              dnu[c] = fmaf(au, cv[5 + c], dnu[c]);
              dnv[c] = fmaf(av, cv[5 + c], dnv[c]);
            }
          }
        }
        const float nt0 = nt01.x, nt1 = nt01.y;
        float dxs = dxy.x, dys = dxy.y;
        // two-component normal: n^t = (n_x, n_y, n_z(n_x, n_y)); dL/d(n_x, n_y)
        // = (e0, e1) + e2 dn_z/d(n_x, n_y), dn_z/dn_x = -n_x / n_z
        float inz = 0.f;
        if (N2) {
          nt2 = rebuild_nz(nt0, nt1);
          inz = nt2 > 0.f ? 1.f / nt2 : 0.f;
          gxx = fmaf(e0, nt0, fmaf(e1, nt1, fmaf(e2, nt2, gxx)));  // dL/dX . x: the normal's share
          const float k = -e2 * inz;
          g8[5] = fmaf(k, nt0, e0);
          g8[6] = fmaf(k, nt1, e1);
          dxs = fmaf(g8[5], dnu[0], fmaf(g8[6], dnu[1], dxs));
          dys = fmaf(g8[5], dnv[0], fmaf(g8[6], dnv[1], dys));
        }
        // indirect light of the fragment: l = c . Y(w_r), w_r the reflection
        // of w_o about normalize(n_w), n_w = [t_u t_v n_f] n^t (Eq. 7)
        // (one pass over the coefficients also gives s_j = dL/dX_ind . c_j
        // and with it the direction gradient gd = sum_j s_j grad Y_j(w_r),
        // both still to be scaled by the fragment's weight)
        float lx = 0.f, ly = 0.f, lz = 0.f;
        Refl rf;
        float3 gd = make_float3(0.f, 0.f, 0.f);
        if (IND && V.sh) {
          const float3 nw = make_float3(fmaf(nt0, r.r2.z, fmaf(nt1, r.r3.y, nt2 * r.r4.x)),
                                        fmaf(nt0, r.r2.w, fmaf(nt1, r.r3.z, nt2 * r.r4.y)),
                                        fmaf(nt0, r.r3.x, fmaf(nt1, r.r3.w, nt2 * r.r4.z)));
          rf = reflect_dir(nw, wo);
          sh_basis(rf.wr, shK, shv + 3);
          float sj[9];
          const float3 l = sh_eval<true>(V.sh + splat * V.sh_stride, shK, shv + 3,
                                         make_float3(gXi[0], gXi[1], gXi[2]), sj);
          gd = sh_grad_dir(rf.wr, shK, sj);
          lx = l.x;
          ly = l.y;
          lz = l.z;
        }
        // dL/dalpha = T_before (Q - P): Q = gX.x + gA of this fragment, P the
        // same projection of everything blended behind it (P <- a Q + (1-a) P)
        const float z = r.r4.w * f.rd;  // camera depth of the hit
        const float Q = fmaf(gXi[0], lx, fmaf(gXi[1], ly, fmaf(gXi[2], lz, fmaf(gZ, z, gxx + gA))));
        const float ga = (Q - P) * Tb;
        P = fmaf(f.alpha, Q, om * P);
        Tcur = Tb;
        {
          const float2 W = f2(wgt, wgt);
          float2 p0 = mul2(W, g01), p1 = mul2(W, g23), p2 = mul2(W, g45), p3 = mul2(W, g67);
          t8[0] = p0.x; t8[1] = p0.y; t8[2] = p1.x; t8[3] = p1.y;
          t8[4] = p2.x; t8[5] = p2.y; t8[6] = p3.x; t8[7] = p3.y;
          if (N2) {
            t8[5] = wgt * g8[5];
            t8[6] = wgt * g8[6];
          }
        }
        dxs *= wgt;
        dys *= wgt;
        float gn0 = wgt * gX[5], gn1 = wgt * gX[6], gn2 = wgt * gX[7];
        if (IND && V.sh) {
          // dL/dl = wgt dL/dX_ind; through w_r into the fragment's normal
          const float d0 = wgt * gXi[0], d1 = wgt * gXi[1], d2 = wgt * gXi[2];
          shv[0] = d0;
          shv[1] = d1;
          shv[2] = d2;
          const float gx = wgt * gd.x, gy = wgt * gd.y, gz = wgt * gd.z;
          // w_r = 2 (n.w_o) n - w_o  ->  dL/dn = 2 ((n.w_o) g + (g.n) w_o)
          const float gdn = gx * rf.nh.x + gy * rf.nh.y + gz * rf.nh.z;
          float en0 = 2.f * (rf.ndw * gx + gdn * wo.x), en1 = 2.f * (rf.ndw * gy + gdn * wo.y);
          float en2 = 2.f * (rf.ndw * gz + gdn * wo.z);
          // n = n_w / |n_w|
          const float pr = en0 * rf.nh.x + en1 * rf.nh.y + en2 * rf.nh.z;
          en0 = (en0 - rf.nh.x * pr) * rf.inl;
          en1 = (en1 - rf.nh.y * pr) * rf.inl;
          en2 = (en2 - rf.nh.z * pr) * rf.inl;
          // into the tangent normal (R'^T e): its texels, the texture
          // coordinates it is interpolated at, and the frame's torque
          float et0 = r.r2.z * en0 + r.r2.w * en1 + r.r3.x * en2;
          float et1 = r.r3.y * en0 + r.r3.z * en1 + r.r3.w * en2;
          float et2 = r.r4.x * en0 + r.r4.y * en1 + r.r4.z * en2;
          if (N2) {  // through the rebuilt n_z into the stored (n_x, n_y)
            const float k = -et2 * inz;
            et0 = fmaf(k, nt0, et0);
            et1 = fmaf(k, nt1, et1);
            et2 = 0.f;
          }
          t8[5] += et0;
          t8[6] += et1;
          t8[7] += et2;
          dxs = fmaf(et0, dnu[0], fmaf(et1, dnu[1], fmaf(et2, dnu[2], dxs)));
          dys = fmaf(et0, dnv[0], fmaf(et1, dnv[1], fmaf(et2, dnv[2], dys)));
          gn0 += en0;
          gn1 += en1;
          gn2 += en2;
        }
        // alpha = min(0.99, o G), G = exp(-(u^2+v^2)/2)
        float go = 0.f, gG = 0.f;
        if (f.oG <= kAlphaMax()) {
          go = ga * f.G;
          gG = ga * r.r2.y;
        }
        const float gu = fmaf(dxs, Ts6, -gG * f.G * f.u);
        const float gv = fmaf(dys, Ts6, -gG * f.G * f.v);
        // u = un / den, v = vn / den
        const float gun = gu * f.rd, gvn = gv * f.rd;
        // z = D / den enters through den and D (dL/dz = wgt gZ)
        const float gzw = wgt * gZ;
        const float gden = -fmaf(gzw, z, gu * f.u + gv * f.v) * f.rd;
        {
          const float2 XY = f2(xp, yp);
          const float2 a0 = mul2(f2(gun, gun), XY), a1 = mul2(f2(gvn, gvn), XY), a2 = mul2(f2(gden, gden), XY);
          gi[0] = a0.x; gi[1] = a0.y; gi[2] = gun;
          gi[3] = a1.x; gi[4] = a1.y; gi[5] = gvn;
          gi[6] = a2.x; gi[7] = a2.y; gi[8] = gden;
        }
        gi[9] = go;
        // normal-mapping frame [t_u t_v n_f]: its gradient is the outer
        // product nt (x) gn per column, but only the frame's rotation reaches
        // the parameters, so the sum over columns of f_a x (nt_a gn) -- the
        // torque n_w x gn with n_w the fragment's world normal (Eq. 7) -- is
        // all that is reduced
        const float nw0 = fmaf(nt0, r.r2.z, fmaf(nt1, r.r3.y, nt2 * r.r4.x));
        const float nw1 = fmaf(nt0, r.r2.w, fmaf(nt1, r.r3.z, nt2 * r.r4.y));
        const float nw2 = fmaf(nt0, r.r3.x, fmaf(nt1, r.r3.w, nt2 * r.r4.z));
        gi[10] = fmaf(nw1, gn2, -nw2 * gn1);
        gi[11] = fmaf(nw2, gn0, -nw0 * gn2);
        gi[12] = fmaf(nw0, gn1, -nw1 * gn0);
        gi[13] = gzw * f.rd;  // dL/dD
      }
      // per-splat record gradients (14 values, padded to 16): a halving
      // reduce-scatter over the warp (16 shuffles); afterwards lane pair
      // (2i, 2i+1) holds the warp's sum of value i and lane 2i adds it
      if (!ok) {
#pragma unroll
        for (int q = 0; q < kRecGrads; ++q) gi[q] = 0.f;
      }
      {
        const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4, u2 = lane & 2;
        float v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = q < kRecGrads ? gi[q] : 0.f;
        float a8[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float snd = u16 ? v[q] : v[8 + q], kp = u16 ? v[8 + q] : v[q];
          a8[q] = kp + __shfl_xor_sync(FULL, snd, 16);
        }
        float a4[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float snd = u8 ? a8[q] : a8[4 + q], kp = u8 ? a8[4 + q] : a8[q];
          a4[q] = kp + __shfl_xor_sync(FULL, snd, 8);
        }
        float a2[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const float snd = u4 ? a4[q] : a4[2 + q], kp = u4 ? a4[2 + q] : a4[q];
          a2[q] = kp + __shfl_xor_sync(FULL, snd, 4);
        }
        const float snd = u2 ? a2[0] : a2[1], kp = u2 ? a2[1] : a2[0];
        float sum = kp + __shfl_xor_sync(FULL, snd, 2);
        sum += __shfl_xor_sync(FULL, sum, 1);
        const int idx = (lane >> 1) & 15;
        if (!(lane & 1) && idx < kRecGrads && sum != 0.f)
          atomicAdd(g_items + (size_t)item * kRecGradStride + idx, (double)sum);
      }
      // SH coefficient gradients of the splat: dL/dc_jc = sum over lanes of
      // (dL/dl_c) Y_j -- lane v < 3K gathers its (c, j) products through
      // shared memory and adds them once per warp
      if (IND && V.sh) {
#pragma unroll
        for (int q = 0; q < 12; ++q) s_sh[IND ? warp : 0][q][lane] = shv[q];
        __syncwarp();
        if (lane < 3 * shK && g.sh) {
          const int j = lane / 3, c = lane - 3 * j;
          const float4* dc = reinterpret_cast<const float4*>(s_sh[IND ? warp : 0][c]);
          const float4* yj = reinterpret_cast<const float4*>(s_sh[IND ? warp : 0][3 + j]);
          float acc = 0.f;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 a = dc[q], b = yj[q];
            acc = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, acc))));
          }
          if (acc != 0.f) red_add(g.sh + splat * 3 * shK + lane, acc);
        }
        __syncwarp();
      }
      // texel gradients: lanes are grouped by bilinear cell (the four texels
      // they interpolate).  A lane whose cell at most kDirect live lanes share
      // adds its own four corners (16-byte vector reductions); each larger
      // group is summed over the warp by one halving reduce-scatter of its
      // 32 values (4 corners x 8 channels, 31 shuffles), after which lane L
      // holds corner L >> 3, channel L & 7 and all 32 lanes issue one
      // reduction covering the cell's four texels.  A warp's live lanes
      // usually share one to three cells.
      if (g.texels) {
        constexpr int kDirect = 8;
        const unsigned key = ok ? (unsigned)(ts_.ia | (ts_.ib << 8) | (ts_.ja << 16) | (ts_.jb << 24)) : FULL;
        float* gtex = g.texels + splat * (long long)T * T * 8;
        if (!ok) {
#pragma unroll
          for (int c = 0; c < 8; ++c) t8[c] = 0.f;
        }
        const unsigned live = __ballot_sync(FULL, ok);
        const unsigned same = __match_any_sync(FULL, key) & live;
        const bool direct = ok && __popc(same) <= kDirect;
        if (__any_sync(FULL, direct) && direct) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int jj = (k & 2) ? ts_.jb : ts_.ja, ii = (k & 1) ? ts_.ib : ts_.ia;
            float* p = gtex + (jj * T + ii) * 8;
            const float2 Wk = f2(w4[k], w4[k]);
            const float2 v0 = mul2(Wk, f2(t8[0], t8[1])), v1 = mul2(Wk, f2(t8[2], t8[3]));
            const float2 v2 = mul2(Wk, f2(t8[4], t8[5])), v3 = mul2(Wk, f2(t8[6], t8[7]));
            red_add_v4(p, v0.x, v0.y, v1.x, v1.y);
            red_add_v4(p + 4, v2.x, v2.y, v3.x, v3.y);
          }
        }
        const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4, u2 = lane & 2, u1 = lane & 1;
        unsigned pend = __ballot_sync(FULL, ok && !direct);
        // lane bit 4 <-> corner bit 1 (row jb), bit 3 <-> corner bit 0
        // (column ib), bits 2..0 <-> channel; each step keeps the half
        // selected by the lane's bit and adds the partner's copy of it.  The
        // corner weights are taken in lane order, wp[j] = w4[c ^ j] with c
        // the corner the lane keeps, so that the two corner steps need no
        // per-value selects
        float wp[4];
        {
          const float r0 = u8 ? w4[1] : w4[0], r1 = u8 ? w4[0] : w4[1];
          const float r2 = u8 ? w4[3] : w4[2], r3 = u8 ? w4[2] : w4[3];
          wp[0] = u16 ? r2 : r0;
          wp[1] = u16 ? r3 : r1;
          wp[2] = u16 ? r0 : r2;
          wp[3] = u16 ? r1 : r3;
        }
        while (pend) {  // warp-uniform
          const unsigned lk = __shfl_sync(FULL, key, __ffs(pend) - 1);
          const bool mem = ((pend >> lane) & 1u) && key == lk;
          pend &= ~__ballot_sync(FULL, mem);
          const float wk0 = mem ? wp[0] : 0.f, wk1 = mem ? wp[1] : 0.f;
          const float ws0 = mem ? wp[2] : 0.f, ws1 = mem ? wp[3] : 0.f;
          const float2 WK0 = f2(wk0, wk0), WK1 = f2(wk1, wk1), WS0 = f2(ws0, ws0), WS1 = f2(ws1, ws1);
          // channel pairs: a[q] = channels (2q, 2q+1) of the lane's own
          // column, a[4+q] of the other column (the partner's own)
          float2 a[8];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float2 t = f2(t8[2 * q], t8[2 * q + 1]);
            const float2 s0 = mul2(WS0, t), s1 = mul2(WS1, t);
            a[q] = fma2(WK0, t, f2(__shfl_xor_sync(FULL, s0.x, 16), __shfl_xor_sync(FULL, s0.y, 16)));
            a[4 + q] = fma2(WK1, t, f2(__shfl_xor_sync(FULL, s1.x, 16), __shfl_xor_sync(FULL, s1.y, 16)));
          }
#pragma unroll
          for (int q = 0; q < 4; ++q)
            a[q] = add2(a[q], f2(__shfl_xor_sync(FULL, a[4 + q].x, 8), __shfl_xor_sync(FULL, a[4 + q].y, 8)));
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const float2 snd = u4 ? a[q] : a[2 + q], kp = u4 ? a[2 + q] : a[q];
            a[q] = add2(kp, f2(__shfl_xor_sync(FULL, snd.x, 4), __shfl_xor_sync(FULL, snd.y, 4)));
          }
          {
            const float2 snd = u2 ? a[0] : a[1], kp = u2 ? a[1] : a[0];
            a[0] = add2(kp, f2(__shfl_xor_sync(FULL, snd.x, 2), __shfl_xor_sync(FULL, snd.y, 2)));
          }
          const float res = (u1 ? a[0].y : a[0].x) + __shfl_xor_sync(FULL, u1 ? a[0].x : a[0].y, 1);
          const int ii = (int)((lk >> (u8 ? 8 : 0)) & 0xffu);
          const int jj = (int)((lk >> (u16 ? 24 : 16)) & 0xffu);
          red_add(gtex + (jj * T + ii) * 8 + (lane & 7), res);
        }
      }
    }
  }
    __syncwarp();
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

void launch_raster_bwd(const ViewTable& vt, const Record* rec, const uint32_t* pair_items,
                       const uint2* ranges, int tex_dtype, const float4* gxa, double* g_items,
                       const GradTable& g, int feat, cudaStream_t st) {
  dim3 grid(vt.n_tiles * kCtasPerTile), block(32 * kRasterWarps);
#define TS_LAUNCH_B(DTV)                                                                                      \
  switch (feat & (FEAT_IND | FEAT_N2)) {                                                                      \
    case 0: k_raster_bwd<DTV, 0><<<grid, block, 0, st>>>(vt, rec, pair_items, ranges, gxa, g_items, g); break; \
    case FEAT_N2:                                                                                             \
      k_raster_bwd<DTV, FEAT_N2><<<grid, block, 0, st>>>(vt, rec, pair_items, ranges, gxa, g_items, g);       \
      break;                                                                                                  \
    case FEAT_IND:                                                                                            \
      k_raster_bwd<DTV, FEAT_IND><<<grid, block, 0, st>>>(vt, rec, pair_items, ranges, gxa, g_items, g);      \
      break;                                                                                                  \
    default:                                                                                                  \
      k_raster_bwd<DTV, FEAT_IND | FEAT_N2><<<grid, block, 0, st>>>(vt, rec, pair_items, ranges, gxa, g_items, \
                                                                    g);                                       \
  }
  if (tex_dtype == DT_F32) {
    TS_LAUNCH_B(DT_F32)
  } else if (tex_dtype == DT_BF16) {
    TS_LAUNCH_B(DT_BF16)
  } else {
    TS_LAUNCH_B(DT_F16)
  }
#undef TS_LAUNCH_B
  note_launches(1);
}

}  // namespace ts
