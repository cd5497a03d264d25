// ts_render_noalloc: one-view forward render that allocates no memory.
//
// For callers that cannot allocate device memory while they render: a
// renderer embedded in a host application that owns the whole device
// budget, a real-time frame loop where an allocation's latency or failure
// is not acceptable, or a plugin that may only touch buffers it was handed.
// Every input and the output are caller buffers; the working set (per-splat
// records, sort keys, pair lists, tile ranges, sort temporaries) lives in
// one file-scope device array of fixed size, so the call never calls
// cudaMalloc / cudaFree or any allocating routine.
//
// The array is shared by every call on a device and keeps the previous
// call's contents; the per-call state that must start at zero (tile ranges)
// is cleared on each call.  Two calls that overlap on the GPU (different
// streams, no ordering between them) race on the array.
#include <cstring>
#include <mutex>
#include <string>

#include "kernels.h"
#include "prof.h"
#include "../../include/texsplat.h"

using namespace ts;

namespace {

// Limits of the fixed working set.
constexpr long long NA_MAX_SPLATS = 32768;
constexpr long long NA_MAX_TILES = 8192;      // e.g. 1920x1080 = 8160 tiles
constexpr long long NA_MAX_PAIRS = 1 << 20;   // (tile, splat) pairs after binning

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Byte layout of the array (each region 256-byte aligned).
constexpr size_t OFF_MEANS = 0;
constexpr size_t OFF_REC = OFF_MEANS + align256(NA_MAX_SPLATS * sizeof(float4));
constexpr size_t OFF_COUNTS = OFF_REC + align256(NA_MAX_SPLATS * sizeof(Record));
constexpr size_t OFF_IDS0 = OFF_COUNTS + align256(NA_MAX_SPLATS * 4);
constexpr size_t OFF_IDS1 = OFF_IDS0 + align256(NA_MAX_SPLATS * 4);
constexpr size_t OFF_CS = OFF_IDS1 + align256(NA_MAX_SPLATS * 4);
constexpr size_t OFF_OFFS = OFF_CS + align256(NA_MAX_SPLATS * 4);
constexpr size_t OFF_DK0 = OFF_OFFS + align256(NA_MAX_SPLATS * 4);
constexpr size_t OFF_DK1 = OFF_DK0 + align256(NA_MAX_SPLATS * 8);
constexpr size_t OFF_RECTS = OFF_DK1 + align256(NA_MAX_SPLATS * 8);
constexpr size_t OFF_TK0 = OFF_RECTS + align256(NA_MAX_SPLATS * sizeof(int4));
constexpr size_t OFF_TK1 = OFF_TK0 + align256(NA_MAX_PAIRS * 4);
constexpr size_t OFF_PI0 = OFF_TK1 + align256(NA_MAX_PAIRS * 4);
constexpr size_t OFF_PI1 = OFF_PI0 + align256(NA_MAX_PAIRS * 4);
constexpr size_t OFF_RANGES = OFF_PI1 + align256(NA_MAX_PAIRS * 4);
constexpr size_t OFF_TEMP = OFF_RANGES + align256(NA_MAX_TILES * sizeof(uint2));
// sort / scan temporaries for up to NA_MAX_PAIRS keys: 256 digit counters
// per 4096-key block, twice, plus the nested scan levels
constexpr size_t TEMP_BYTES = 2 * 256 * 256 * 4 + 64 * 1024;
constexpr size_t NA_BYTES = OFF_TEMP + align256(TEMP_BYTES);

}  // namespace

// The working set: about 21 MB, resident on every device that loads the library.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

namespace {

std::mutex g_na_mu;
void* g_na_ptr[64] = {nullptr};

// failures are reported through ts_last_error() like every other entry point
ts_status na_fail(ts_status code, const std::string& msg) { return ts::set_error(code, msg); }

}  // namespace

extern "C" ts_status ts_render_noalloc(int64_t n, const float* means, const float* quats, const float* scales,
                                       const float* opacity, int T, const float* texels, int levels, int base_res,
                                       const float* spec, int irr_res, const float* irr, int lut_res,
                                       const float* lut, const ts_camera* cam, float* out_rgba, void* stream) {
  if (!cam || !out_rgba) return na_fail(TS_ERR_ARG, "ts_render_noalloc: NULL camera or output");
  if (n < 0 || n > NA_MAX_SPLATS) return na_fail(TS_ERR_CAPACITY, "ts_render_noalloc: n exceeds 32768 splats");
  if (n > 0 && (!means || !quats || !scales || !opacity || !texels))
    return na_fail(TS_ERR_ARG, "ts_render_noalloc: NULL splat array");
  if ((reinterpret_cast<uintptr_t>(quats) & 15) || (reinterpret_cast<uintptr_t>(texels) & 15) ||
      (reinterpret_cast<uintptr_t>(scales) & 7))
    return na_fail(TS_ERR_ARG, "ts_render_noalloc: quats/texels need 16-byte, scales 8-byte alignment");
  if (T < 1 || T > 32) return na_fail(TS_ERR_ARG, "ts_render_noalloc: T must be in [1, 32]");
  if (levels < 1 || levels > MAX_LEVELS || base_res < 1 || irr_res < 1 || lut_res < 1 || !spec || !irr || !lut)
    return na_fail(TS_ERR_ARG, "ts_render_noalloc: bad environment");
  if (cam->width < 1 || cam->height < 1 || !(cam->fx > 0.f) || !(cam->fy > 0.f))
    return na_fail(TS_ERR_ARG, "ts_render_noalloc: bad camera");
  const long long tiles_x = (cam->width + TILE - 1) / TILE, tiles_y = (cam->height + TILE - 1) / TILE;
  if (tiles_x * tiles_y > NA_MAX_TILES) return na_fail(TS_ERR_CAPACITY, "ts_render_noalloc: more than 8192 tiles");

  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) return na_fail(TS_ERR_CUDA, "ts_render_noalloc: cudaGetDevice failed");
  unsigned char* base = nullptr;
  {
    // set-up, once per device, with that device current
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess)
        return na_fail(TS_ERR_CUDA, std::string("ts_render_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_na_ptr[dev] = p;
    }
    base = static_cast<unsigned char*>(g_na_ptr[dev]);
  }
  auto at = [&](size_t off) { return base + off; };

  ViewTable vt;
  memset(&vt, 0, sizeof(vt));
  vt.n_views = 1;
  ViewDesc& V = vt.v[0];
  memcpy(V.R, cam->R, sizeof(V.R));
  memcpy(V.t, cam->t, sizeof(V.t));
  V.fx = cam->fx; V.fy = cam->fy; V.cx = cam->cx; V.cy = cam->cy;
  V.W = cam->width; V.H = cam->height;
  V.tiles_x = (int)tiles_x; V.tiles_y = (int)tiles_y;
  V.n_splats = (int)n;
  V.means = reinterpret_cast<const float4*>(at(OFF_MEANS));
  V.quats = reinterpret_cast<const float4*>(quats);
  V.scales = reinterpret_cast<const float2*>(scales);
  V.opacity = opacity;
  V.texels = texels;
  V.T = T;
  V.tex_dtype = DT_F32;
  V.tex_v8 = (reinterpret_cast<uintptr_t>(texels) & 31) == 0;
  size_t off = 0;
  for (int l = 0; l < levels; ++l) {
    const int r = base_res >> l > 0 ? base_res >> l : 1;
    V.env.spec[l] = spec + off;
    V.env.spec_res[l] = r;
    off += (size_t)6 * r * r * 3;
  }
  V.env.levels = levels;
  V.env.irr = irr;
  V.env.irr_res = irr_res;
  V.env.cube_dtype = DT_F32;
  V.env.lut = lut;
  V.env.lut_res = lut_res;
  V.rgba = reinterpret_cast<float4*>(out_rgba);
  vt.n_tiles = (int)(tiles_x * tiles_y);
  vt.n_items = (int)n;

  Record* rec = reinterpret_cast<Record*>(at(OFF_REC));
  uint32_t* counts = reinterpret_cast<uint32_t*>(at(OFF_COUNTS));
  uint32_t* ids0 = reinterpret_cast<uint32_t*>(at(OFF_IDS0));
  uint32_t* ids1 = reinterpret_cast<uint32_t*>(at(OFF_IDS1));
  uint32_t* cs = reinterpret_cast<uint32_t*>(at(OFF_CS));
  uint32_t* offs = reinterpret_cast<uint32_t*>(at(OFF_OFFS));
  uint64_t* dk0 = reinterpret_cast<uint64_t*>(at(OFF_DK0));
  uint64_t* dk1 = reinterpret_cast<uint64_t*>(at(OFF_DK1));
  int4* rects = reinterpret_cast<int4*>(at(OFF_RECTS));
  uint32_t* tk0 = reinterpret_cast<uint32_t*>(at(OFF_TK0));
  uint32_t* tk1 = reinterpret_cast<uint32_t*>(at(OFF_TK1));
  uint32_t* pi0 = reinterpret_cast<uint32_t*>(at(OFF_PI0));
  uint32_t* pi1 = reinterpret_cast<uint32_t*>(at(OFF_PI1));
  uint2* ranges = reinterpret_cast<uint2*>(at(OFF_RANGES));
  void* temp = at(OFF_TEMP);

  if (radix_temp_bytes((int)n, 8) > TEMP_BYTES) return na_fail(TS_ERR_CAPACITY, "ts_render_noalloc: sort temporaries");
  if (n > 0) launch_pad4(means, 3, const_cast<float4*>(V.means), n, st);
  launch_preprocess(vt, rec, counts, dk0, ids0, rects, st);
  const int which = radix_sort_u64(dk0, ids0, dk1, ids1, (int)n, 0, 32, temp, st);
  uint32_t* order = which ? ids1 : ids0;
  launch_gather_counts(order, counts, cs, (int)n, st);
  launch_exclusive_scan(cs, offs, (int)n, temp, st);
  // one synchronisation: the pair count and the sort flags (their device
  // words are module variables too, so reading them allocates nothing)
  int* d_flags = sort_error_flag(dev);
  if (!d_flags) return na_fail(TS_ERR_CUDA, "ts_render_noalloc: sort flag lookup failed");
  vt.sort_err = d_flags;
  uint32_t tail[2] = {0, 0};
  int flags[2] = {0, 0};
  e = cudaMemcpyAsync(flags, d_flags, sizeof(flags), cudaMemcpyDeviceToHost, st);
  if (n > 0) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(&tail[0], offs + (n - 1), 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&tail[1], cs + (n - 1), 4, cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess)
    return na_fail(TS_ERR_CUDA, std::string("ts_render_noalloc: pair count: ") + cudaGetErrorString(e));
  if (flags[SORT_FLAG_LISTS]) {  // the depth sort's bounded wait ran out: the lists are not trusted
    cudaMemsetAsync(d_flags, 0, sizeof(flags), st);
    return na_fail(TS_ERR_TIMEOUT, "ts_render_noalloc: a radix-sort look-back wait ran out");
  }
  if (flags[SORT_FLAG_ORDER]) {  // an earlier call's launch order (same result either way)
    e = cudaMemsetAsync(d_flags + SORT_FLAG_ORDER, 0, sizeof(int), st);
    if (e != cudaSuccess) return na_fail(TS_ERR_CUDA, std::string("ts_render_noalloc: ") + cudaGetErrorString(e));
  }
  const long long K = (long long)tail[0] + tail[1];
  if (K > NA_MAX_PAIRS) return na_fail(TS_ERR_CAPACITY, "ts_render_noalloc: more than 1048576 (tile, splat) pairs");
  if (radix_temp_bytes((int)K, 4) > TEMP_BYTES) return na_fail(TS_ERR_CAPACITY, "ts_render_noalloc: sort temporaries");
  launch_emit_pairs(vt, order, offs, cs, rects, tk0, pi0, (int)n, st);
  int tb = 1;
  while ((1ll << tb) < vt.n_tiles) ++tb;
  const int w2 = radix_sort_u32(tk0, pi0, tk1, pi1, (int)K, 0, tb, temp, st, -1);
  uint32_t* tkeys = w2 ? tk1 : tk0;
  uint32_t* pitems = w2 ? pi1 : pi0;
  e = cudaMemsetAsync(ranges, 0, (size_t)vt.n_tiles * sizeof(uint2), st);
  if (e != cudaSuccess) return na_fail(TS_ERR_CUDA, std::string("ts_render_noalloc: ") + cudaGetErrorString(e));
  launch_tile_ranges(tkeys, (int)K, vt.n_tiles, ranges, st);
  // tile launch order in the pair-key buffer the sort left free (4 x tiles <= pairs capacity)
  static_assert(4 * NA_MAX_TILES <= NA_MAX_PAIRS, "tile order buffer");
  if (radix_temp_bytes(vt.n_tiles, 4) > TEMP_BYTES) return na_fail(TS_ERR_CAPACITY, "ts_render_noalloc: sort temporaries");
  vt.tile_order = launch_tile_order(ranges, vt.n_tiles, w2 ? tk0 : tk1, temp, st);
  launch_raster_fwd(vt, rec, pitems, ranges, DT_F32, false, nullptr, SMP_SOFTWARE, 0, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(TS_ERR_CUDA, std::string("ts_render_noalloc: launch: ") + cudaGetErrorString(e));
  return TS_OK;
}
