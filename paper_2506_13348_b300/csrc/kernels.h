// Host-side launch wrappers of the renderer's kernels.
#pragma once
#include <string>

#include "ts_common.cuh"

namespace ts {

struct GradTable {
  float* means;
  float* quats;
  float* scales;
  float* opacity;
  float* texels;
  float* spec[MAX_LEVELS];
  float* irr;
  float* sh;  // [n][K][3] SH coefficients of the indirect light, or NULL
};

// api.cu: records the message returned by ts_last_error() and returns code
int set_error(int code, const std::string& msg);
}  // namespace ts

struct ts_scene;
struct ts_camera;
struct ts_saved;

namespace ts {
// api.cu: ts_render_views with an admission hook.  After its one
// synchronisation, once the batch's pair count K is known and before any
// per-pair buffer is allocated, reserve(ctx, bytes, K) is called with the
// device bytes the rest of the call allocates; a status other than TS_OK
// ends the call with that status (nothing of the batch is left allocated).
typedef int (*ReserveFn)(void* ctx, size_t bytes, long long pairs);
int render_views_hooked(ts_scene* const* scenes, const ts_camera* cams, int n_views, float* const* out_rgba,
                        ts_saved** saved_out, void* stream, ReserveFn reserve, void* ctx);
// Device bytes ts_render_views allocates before that synchronisation for
// n_items (view, splat) items.
size_t render_views_fixed_bytes(long long n_items);

// preprocess.cu
void launch_preprocess(const ViewTable& vt, Record* rec, uint32_t* counts, uint64_t* depth_keys,
                       uint32_t* item_ids, int4* rects, cudaStream_t st);
void launch_preprocess_bwd(const ViewTable& vt, const double* g_items, const GradTable& g, cudaStream_t st);

// sort.cu
size_t scan_temp_bytes(int n);
void launch_exclusive_scan(const uint32_t* in, uint32_t* out, int n, void* temp, cudaStream_t st);
size_t radix_temp_bytes(int n, int key_bytes);  // temporaries of a sort of n keys of key_bytes (4 or 8)
// Per-device flags (two device ints, 0 while no sort failed) set when a
// bounded look-back wait of a sort ran out: word SORT_FLAG_LISTS for the
// depth sort (and consumers that found an id out of range), word
// SORT_FLAG_ORDER for the rasterisers' launch-order sorts.  The host reads
// and clears them.
int* sort_error_flag(int device);
int sort_wait_selftest(cudaStream_t st);
// Stable LSD radix sort of (key, value) pairs over key bits [begin_bit, end_bit).
// Ping-pongs between (k0, v0) and (k1, v1); returns 0 if the result is in
// (k0, v0), 1 if in (k1, v1).
int radix_sort_u64(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int n, int begin_bit, int end_bit,
                   void* temp, cudaStream_t st);
// flag_word: SORT_FLAG_LISTS / SORT_FLAG_ORDER allow the one-kernel-per-pass
// sort with a bounded wait for n <= 2^18 (a wait that runs out raises that
// word); -1 always takes the separate histogram / scan / scatter passes,
// which wait on nothing (the pair and chart-order sorts).
int radix_sort_u32(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, int n, int begin_bit, int end_bit,
                   void* temp, cudaStream_t st, int flag_word);
void launch_sum_counts(const uint32_t* counts, int n, unsigned long long* total, cudaStream_t st);
void launch_gather_counts(const uint32_t* order, const uint32_t* counts, uint32_t* counts_sorted, int n,
                          cudaStream_t st);
void launch_emit_pairs(const ViewTable& vt, const uint32_t* order, const uint32_t* offsets,
                       const uint32_t* counts_sorted, const int4* rects, uint32_t* tile_keys,
                       uint32_t* pair_items, int n, cudaStream_t st);
void launch_tile_ranges(const uint32_t* tile_keys, int K, int n_tiles, uint2* ranges, cudaStream_t st);
// Tile launch order, longest list first: buf holds 4 * n words (keys and ids,
// twice); returns the n sorted tile ids (inside buf).  temp: radix_temp_bytes(n, 4).
const uint32_t* launch_tile_order(const uint2* ranges, int n, uint32_t* buf, void* temp, cudaStream_t st);
// The same for the backward, by the entries it walks (up to each pixel's last
// blended entry, vt.v[].last); 256-thread CTAs assume TILE == 16.
const uint32_t* launch_tile_order_walk(const ViewTable& vt, const uint2* ranges, uint32_t* buf, void* temp,
                                       cudaStream_t st);
void launch_depth_bits(const uint64_t* depth_keys_unsorted, uint32_t* out, int n, cudaStream_t st);

// raster_fwd.cu / raster_bwd.cu
// Counters of the statistics pass (a forward that writes only these):
// counts[0] evaluated, counts[1] blended fragments; touched is a bitmap with
// words_per_item 32-bit words per list item, bit j T + i set when a blended
// fragment of the item reads texel (i, j) (its four bilinear corners).
struct FragCounters {
  unsigned long long* counts;
  uint32_t* touched;
  int words_per_item;
};
void launch_raster_fwd(const ViewTable& vt, const Record* rec, const uint32_t* pair_items,
                       const uint2* ranges, int tex_dtype, bool save, const FragCounters* stats, int sampler,
                       int feat, cudaStream_t st);
// counts[2] += set bits of the bitmap, counts[3] += items with any bit set
void launch_touch_counts(const uint32_t* touched, long long n_items, int words_per_item, unsigned long long* counts,
                         cudaStream_t st);
void launch_pack_atlas2d(const void* texels, int dtype, long long n, int T, int charts_x, cudaSurfaceObject_t s0,
                         cudaSurfaceObject_t s1, uint2* chart, const uint32_t* chart_of, int half_store,
                         cudaStream_t st);
void launch_morton_order(const float4* means, long long n, uint32_t* bbox, uint32_t* codes, uint32_t* ids,
                         cudaStream_t st);
void launch_chart_of(const uint32_t* ids_sorted, long long n, uint32_t* chart_of, cudaStream_t st);
void launch_raster_bwd(const ViewTable& vt, const Record* rec, const uint32_t* pair_items,
                       const uint2* ranges, int tex_dtype, const float4* gxa, double* g_items,
                       const GradTable& g, int feat, cudaStream_t st);
// shade_bwd.cu: per-pixel shading adjoint -> gxa [pixels][3] (dL/dX 0-3, 4-7, dL/dA)
void launch_shade_bwd(const ViewTable& vt, float4* gxa, const GradTable& g, cudaStream_t st);

// optim.cu
void launch_adam(float* p, float* g, float* m, float* v, long long n, float lr, float b1, float b2, float eps,
                 long long step, void* shadow, int shadow_dtype, int zero_grad, cudaStream_t st);

// misc.cu
void launch_pack_texels(const float* src, void* dst, long long n, int dtype, cudaStream_t st);
void launch_activate(const float* log_s, const float* logit_o, long long n, float* s, float* o, cudaStream_t st);
void launch_activate_bwd(const float* s, const float* o, const float* gs, const float* go, long long n,
                         float* g_log_s, float* g_logit_o, int accumulate, cudaStream_t st);
void launch_pack_f16(const float* src, __half* dst, long long n, cudaStream_t st);
void launch_pad4(const float* src, int comps, float4* dst, long long n, cudaStream_t st);
// out: 3 device words, initialised to {0, 0xffffffff, 0} by the caller
void launch_validate_gaussians(const float4* means, const float4* quats, const float2* scales, const float* opac,
                               long long n, unsigned* out, cudaStream_t st);
void launch_l1_loss(const float4* rgba, const float4* target, long long n, float* loss, float4* grad,
                    cudaStream_t st);

// loss.cu: image term of the training loss (L1 + D-SSIM)
int set_gauss_window(int device);
size_t image_loss_temp_bytes(int W, int H);
void launch_image_loss(const float4* img, const float4* tgt, int W, int H, float lam, float* loss, float4* grad,
                       void* temp, cudaStream_t st);

// normal_loss.cu: normal consistency against the depth-derived normal
size_t normal_loss_temp_bytes(int W, int H);
void launch_normal_loss(const ViewDesc& V, float weight, float* loss, float4* gnorm, float* gzsum, void* temp,
                        cudaStream_t st);

}  // namespace ts
