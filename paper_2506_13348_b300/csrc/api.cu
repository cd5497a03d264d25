// C ABI of the textured 2DGS renderer: scene memory, the render / backward
// launch sequences and inspection helpers.  See include/texsplat.h.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.h"
#include "prof.h"
#include "../../include/texsplat.h"

using namespace ts;

namespace {

thread_local std::string g_err;

ts_status fail(ts_status code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define TS_CUDA(call)                                                                              \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) {                                                                       \
      return fail(e_ == cudaErrorMemoryAllocation ? TS_ERR_OOM : TS_ERR_CUDA,                      \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                             \
    }                                                                                              \
  } while (0)

#define TS_CHECK_LAUNCH()                                                                          \
  do {                                                                                             \
    cudaError_t e_ = cudaGetLastError();                                                           \
    if (e_ != cudaSuccess) return fail(TS_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
  } while (0)

// Host-side failure injection for tests: when armed with k >= 0, the
// (k+1)-th device allocation the library makes from then on fails with
// cudaErrorMemoryAllocation (once), as a real out-of-memory would.
std::atomic<long long> g_fail_alloc{-1};
bool injected_failure() {
  long long k = g_fail_alloc.load();
  while (k >= 0) {
    if (g_fail_alloc.compare_exchange_weak(k, k - 1)) return k == 0;
  }
  return false;
}
cudaError_t dev_malloc(void** p, size_t bytes) {
  if (injected_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}
cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t st) {
  if (injected_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocAsync(p, bytes, st);
}

std::mutex g_pool_mu;
bool g_pool_set[64] = {false};

ts_status prepare_device(int device) {
  TS_CUDA(cudaSetDevice(device));
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (device >= 0 && device < 64 && !g_pool_set[device]) {
    cudaMemPool_t pool;
    TS_CUDA(cudaDeviceGetDefaultMemPool(&pool, device));
    uint64_t thr = UINT64_MAX;
    TS_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    g_pool_set[device] = true;
  }
  return TS_OK;
}

// Stream-ordered scratch allocations released together.
struct Scratch {
  cudaStream_t st;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t s) : st(s) {}
  cudaError_t alloc(void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = dev_malloc_async(p, bytes, st);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
  void release() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
    ptrs.clear();
  }
  ~Scratch() { release(); }
};

int bits_for(long long n) {
  int b = 0;
  while ((1ll << b) < n) ++b;
  return b;
}

}  // namespace

struct ts_scene {
  int device = 0;
  int64_t n = 0;
  float4* means = nullptr;
  float4* quats = nullptr;
  float2* scales = nullptr;
  float* opacity = nullptr;
  void* texels = nullptr;
  int T = 0;
  int tex_dtype = 0;
  int64_t tex_n = -1;
  void* spec = nullptr;  // all levels, concatenated
  size_t spec_off[MAX_LEVELS] = {0};
  int spec_res[MAX_LEVELS] = {0};
  int levels = 0;
  void* irr = nullptr;
  int irr_res = 0;
  int cube_dtype = 0;
  float* lut = nullptr;
  int lut_res = 0;
  int64_t tex_version = 0;  // bumped by every ts_upload_atlas
  int64_t gen = 0;          // bumped whenever an upload replaces (and frees) device buffers
  // 2-D hardware-texture atlases (supplementary Sec. 1) and the indirection buffer
  cudaArray_t a2d[2] = {nullptr, nullptr};
  cudaTextureObject_t a2d_tex[2] = {0, 0};
  uint2* chart = nullptr;
  int64_t a2d_version = -1;  // tex_version the 2-D atlases were built from
  int64_t a2d_n = -1;
  int sampler = SMP_SOFTWARE;
  // indirect light: SH coefficients [n][sh_stride] (K x 3 floats, padded to 4)
  float* sh = nullptr;
  int sh_deg = -1, sh_stride = 0;
  int64_t sh_n = -1;
  bool normal_xy = false;  // two-component tangent normals (Sec. 3.5.1)
};

struct ts_saved {
  int device = 0;
  bool indirect = false;  // the batch blended per-splat SH light
  int feat = 0;           // FEAT_* bits the batch was rendered with
  cudaStream_t stream = nullptr;
  ViewTable vt;
  std::vector<ts_scene*> scenes;
  Record* rec = nullptr;
  uint32_t* pair_items = nullptr;
  uint32_t* tile_keys = nullptr;
  uint2* ranges = nullptr;
  uint32_t* depth_bits = nullptr;
  std::vector<void*> bufs;  // owned, cudaMallocAsync'ed on `stream`
  int64_t K = 0;
  std::vector<int64_t> gens;  // each view's scene generation at the forward
};

namespace {
// The saved state keeps pointers into its scenes' buffers: a backward (or a
// recount) after an upload replaced them would read freed memory.
bool scenes_unchanged(const ts_saved* sv) {
  for (size_t i = 0; i < sv->scenes.size(); ++i)
    if (i >= sv->gens.size() || sv->scenes[i]->gen != sv->gens[i]) return false;
  return true;
}
}  // namespace

int ts::set_error(int code, const std::string& msg) { return fail(code, msg); }

static void free_atlas2d(ts_scene* s) {
  for (int i = 0; i < 2; ++i) {
    if (s->a2d_tex[i]) cudaDestroyTextureObject(s->a2d_tex[i]);
    if (s->a2d[i]) cudaFreeArray(s->a2d[i]);
    s->a2d_tex[i] = 0;
    s->a2d[i] = nullptr;
  }
  if (s->chart) cudaFree(s->chart);
  s->chart = nullptr;
  s->a2d_version = -1;
  s->a2d_n = -1;
}

static void free_scene_buffers(ts_scene* s) {
  void* ptrs[] = {s->means, s->quats, s->scales, s->opacity, s->texels, s->spec, s->irr, s->lut, s->sh};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  free_atlas2d(s);
}

extern "C" {

const char* ts_last_error(void) { return g_err.c_str(); }
const char* ts_version(void) { return "texsplat-b300 0.1 (sm_103a)"; }

ts_status ts_create_scene(ts_scene** out, int device) {
  if (!out) return fail(TS_ERR_ARG, "ts_create_scene: out is NULL");
  int count = 0;
  TS_CUDA(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count) return fail(TS_ERR_ARG, "ts_create_scene: bad device index");
  ts_status st = prepare_device(device);
  if (st != TS_OK) return st;
  ts_scene* s = new (std::nothrow) ts_scene();
  if (!s) return fail(TS_ERR_OOM, "ts_create_scene: host allocation failed");
  s->device = device;
  *out = s;
  return TS_OK;
}

ts_status ts_destroy_scene(ts_scene* s) {
  if (!s) return TS_OK;
  cudaSetDevice(s->device);
  cudaDeviceSynchronize();
  free_scene_buffers(s);
  delete s;
  return TS_OK;
}


// Device buffers of one upload, freed unless released into the scene.
struct UploadBufs {
  std::vector<void*> p;
  cudaError_t alloc(void** out, size_t bytes) {
    cudaError_t e = dev_malloc(out, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess) p.push_back(*out);
    return e;
  }
  void release() { p.clear(); }
  ~UploadBufs() {
    for (void* q : p) cudaFree(q);
  }
};

#define TS_UP(call)                                                                                \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) {                                                                       \
      cudaStreamSynchronize(st);                                                                   \
      return fail(e_ == cudaErrorMemoryAllocation ? TS_ERR_OOM : TS_ERR_CUDA,                      \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                             \
    }                                                                                              \
  } while (0)

ts_status ts_upload_gaussians(ts_scene* s, int64_t n, const float* means, const float* quats, const float* scales,
                              const float* opacity, int src_on_device, void* stream) {
  if (!s) return fail(TS_ERR_ARG, "ts_upload_gaussians: scene is NULL");
  if (n < 0 || n > (int64_t)INT32_MAX / 64) return fail(TS_ERR_ARG, "ts_upload_gaussians: bad n");
  if (n > 0 && (!means || !quats || !scales || !opacity))
    return fail(TS_ERR_ARG, "ts_upload_gaussians: NULL array");
  cudaStream_t st = (cudaStream_t)stream;
  TS_CUDA(cudaSetDevice(s->device));
  TS_CUDA(cudaStreamSynchronize(st));
  // the new buffers are filled and checked before they replace the old ones:
  // a failed upload leaves the scene as it was
  const size_t nn = (size_t)std::max<int64_t>(n, 1);
  UploadBufs b;
  float4 *m4 = nullptr, *q4 = nullptr;
  float2* s2 = nullptr;
  float *o1 = nullptr, *staging = nullptr;
  unsigned* check = nullptr;
  TS_UP(b.alloc((void**)&m4, nn * sizeof(float4)));
  TS_UP(b.alloc((void**)&q4, nn * sizeof(float4)));
  TS_UP(b.alloc((void**)&s2, nn * sizeof(float2)));
  TS_UP(b.alloc((void**)&o1, nn * sizeof(float)));
  TS_UP(b.alloc((void**)&staging, nn * 3 * sizeof(float)));
  TS_UP(b.alloc((void**)&check, 4 * sizeof(unsigned)));
  unsigned res[3] = {0u, 0xffffffffu, 0u};
  TS_UP(cudaMemcpyAsync(check, res, sizeof(res), cudaMemcpyHostToDevice, st));
  if (n > 0) {
    const cudaMemcpyKind kind = src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    TS_UP(cudaMemcpyAsync(staging, means, (size_t)n * 3 * sizeof(float), kind, st));
    launch_pad4(staging, 3, m4, n, st);
    TS_UP(cudaMemcpyAsync(q4, quats, (size_t)n * 4 * sizeof(float), kind, st));
    TS_UP(cudaMemcpyAsync(s2, scales, (size_t)n * 2 * sizeof(float), kind, st));
    TS_UP(cudaMemcpyAsync(o1, opacity, (size_t)n * sizeof(float), kind, st));
    launch_validate_gaussians(m4, q4, s2, o1, n, check, st);
    TS_UP(cudaGetLastError());
    TS_UP(cudaMemcpyAsync(res, check, sizeof(res), cudaMemcpyDeviceToHost, st));
  }
  TS_UP(cudaStreamSynchronize(st));
  if (res[0]) {
    std::string why;
    if (res[2] & 1u) why += " non-finite centre;";
    if (res[2] & 2u) why += " quaternion non-finite or of zero length;";
    if (res[2] & 4u) why += " scale non-finite or <= 0;";
    if (res[2] & 8u) why += " opacity outside [0, 1] or NaN;";
    return fail(TS_ERR_ARG, "ts_upload_gaussians: " + std::to_string(res[0]) + " invalid splat(s), first index " +
                                std::to_string(res[1]) + ":" + why + " the scene is unchanged");
  }
  for (void* p : {(void*)s->means, (void*)s->quats, (void*)s->scales, (void*)s->opacity})
    if (p) cudaFree(p);
  s->gen += 1;
  s->means = m4;
  s->quats = q4;
  s->scales = s2;
  s->opacity = o1;
  s->n = n;
  cudaFree(staging);
  cudaFree(check);
  b.release();
  return TS_OK;
}

ts_status ts_upload_atlas(ts_scene* s, int T, int C, ts_dtype store, const float* texels, int src_on_device,
                          void* stream) {
  if (!s) return fail(TS_ERR_ARG, "ts_upload_atlas: scene is NULL");
  if (C != 8) return fail(TS_ERR_ARG, "ts_upload_atlas: C must be 8");
  if (T < 1 || T > 32) return fail(TS_ERR_ARG, "ts_upload_atlas: T must be in [1, 32]");
  if (store != TS_F32 && store != TS_BF16 && store != TS_F16) return fail(TS_ERR_ARG, "ts_upload_atlas: bad dtype");
  if (s->n > 0 && !texels) return fail(TS_ERR_ARG, "ts_upload_atlas: texels is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  TS_CUDA(cudaSetDevice(s->device));
  TS_CUDA(cudaStreamSynchronize(st));
  const long long count = (long long)s->n * T * T * 8;
  const size_t esz = store == TS_F32 ? 4 : 2;
  UploadBufs b;
  void* tex = nullptr;
  float* staging = nullptr;
  TS_UP(b.alloc(&tex, (size_t)count * esz));
  if (count > 0) {
    if (store == TS_F32) {
      TS_UP(cudaMemcpyAsync(tex, texels, (size_t)count * 4,
                            src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    } else {
      const float* src = texels;
      if (!src_on_device) {
        TS_UP(b.alloc((void**)&staging, (size_t)count * 4));
        TS_UP(cudaMemcpyAsync(staging, texels, (size_t)count * 4, cudaMemcpyHostToDevice, st));
        src = staging;
      }
      {
        ProfScope p(st, "atlas_pack");
        launch_pack_texels(src, tex, count, (int)store, st);
      }
      TS_UP(cudaGetLastError());
    }
  }
  TS_UP(cudaStreamSynchronize(st));
  if (s->texels) cudaFree(s->texels);
  s->gen += 1;
  s->texels = tex;
  s->tex_version += 1;  // any 2-D atlas built from the old texels is stale
  s->T = T;
  s->tex_dtype = (int)store;
  s->tex_n = s->n;
  if (staging) cudaFree(staging);
  b.release();
  return TS_OK;
}

ts_status ts_upload_envmap(ts_scene* s, int levels, int base_res, const float* spec, int irr_res, const float* irr,
                           int lut_res, const float* lut, ts_dtype store, int src_on_device, void* stream) {
  if (!s) return fail(TS_ERR_ARG, "ts_upload_envmap: scene is NULL");
  if (levels < 1 || levels > MAX_LEVELS || base_res < 1 || irr_res < 1 || lut_res < 1)
    return fail(TS_ERR_ARG, "ts_upload_envmap: bad sizes");
  if (!spec || !irr || !lut) return fail(TS_ERR_ARG, "ts_upload_envmap: NULL array");
  if (store != TS_F32 && store != TS_F16) return fail(TS_ERR_ARG, "ts_upload_envmap: store must be F32 or F16");
  cudaStream_t st = (cudaStream_t)stream;
  TS_CUDA(cudaSetDevice(s->device));
  TS_CUDA(cudaStreamSynchronize(st));
  size_t total = 0;
  size_t off[MAX_LEVELS];
  int res[MAX_LEVELS];
  for (int l = 0; l < levels; ++l) {
    res[l] = std::max(1, base_res >> l);
    off[l] = total;
    total += (size_t)6 * res[l] * res[l] * 3;
  }
  const size_t esz = store == TS_F32 ? 4 : 2;
  const size_t irr_n = (size_t)6 * irr_res * irr_res * 3;
  const size_t lut_b = (size_t)lut_res * lut_res * 2 * sizeof(float);
  const cudaMemcpyKind kind = src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  UploadBufs b;
  void *d_spec = nullptr, *d_irr = nullptr;
  float *d_lut = nullptr, *staging = nullptr;
  TS_UP(b.alloc(&d_spec, total * esz));
  TS_UP(b.alloc(&d_irr, irr_n * esz));
  TS_UP(b.alloc((void**)&d_lut, lut_b));
  TS_UP(cudaMemcpyAsync(d_lut, lut, lut_b, kind, st));
  if (store == TS_F32) {
    TS_UP(cudaMemcpyAsync(d_spec, spec, total * 4, kind, st));
    TS_UP(cudaMemcpyAsync(d_irr, irr, irr_n * 4, kind, st));
  } else {
    TS_UP(b.alloc((void**)&staging, (total + irr_n) * 4));
    TS_UP(cudaMemcpyAsync(staging, spec, total * 4, kind, st));
    TS_UP(cudaMemcpyAsync(staging + total, irr, irr_n * 4, kind, st));
    launch_pack_texels(staging, d_spec, (long long)total, DT_F16, st);
    launch_pack_texels(staging + total, d_irr, (long long)irr_n, DT_F16, st);
    TS_UP(cudaGetLastError());
  }
  TS_UP(cudaStreamSynchronize(st));
  for (void* p : {s->spec, s->irr, (void*)s->lut})
    if (p) cudaFree(p);
  s->gen += 1;
  s->spec = d_spec;
  s->irr = d_irr;
  s->lut = d_lut;
  for (int l = 0; l < levels; ++l) {
    s->spec_res[l] = res[l];
    s->spec_off[l] = off[l];
  }
  s->levels = levels;
  s->irr_res = irr_res;
  s->lut_res = lut_res;
  s->cube_dtype = (int)store;
  if (staging) cudaFree(staging);
  b.release();
  return TS_OK;
}

static void fill_env(const ts_scene* s, EnvDesc& E) {
  const size_t esz = s->cube_dtype == DT_F32 ? 4 : 2;
  memset(&E, 0, sizeof(E));
  for (int l = 0; l < s->levels; ++l) {
    E.spec[l] = reinterpret_cast<const char*>(s->spec) + s->spec_off[l] * esz;
    E.spec_res[l] = s->spec_res[l];
  }
  E.levels = s->levels;
  E.irr = s->irr;
  E.irr_res = s->irr_res;
  E.cube_dtype = s->cube_dtype;
  E.lut = s->lut;
  E.lut_res = s->lut_res;
}

static ts_status check_scene(const ts_scene* s) {
  if (!s) return fail(TS_ERR_ARG, "scene is NULL");
  if (!s->means) return fail(TS_ERR_STATE, "geometry not uploaded");
  if (!s->texels || s->tex_n != s->n) return fail(TS_ERR_STATE, "atlas missing or stale (re-upload after geometry)");
  if (!s->spec) return fail(TS_ERR_STATE, "environment not uploaded");
  return TS_OK;
}

static ts_status check_cam(const ts_camera* c) {
  if (!c) return fail(TS_ERR_ARG, "camera is NULL");
  if (c->width < 1 || c->height < 1 || c->width > 16384 || c->height > 16384)
    return fail(TS_ERR_ARG, "camera resolution out of range");
  if (!(c->fx > 0.f) || !(c->fy > 0.f)) return fail(TS_ERR_ARG, "camera focal length must be > 0");
  return TS_OK;
}

}  // extern "C"

// Device bytes ts_render_views allocates before its synchronisation for a
// batch of n_items (view, splat) items: records, counts, ids, offsets,
// depth keys, tile rectangles and the sort / scan temporaries.
size_t ts::render_views_fixed_bytes(long long n_items) {
  const size_t ni = (size_t)std::max<long long>(n_items, 1);
  const size_t rt = std::max(radix_temp_bytes((int)ni, 8), scan_temp_bytes((int)ni));
  return ni * (sizeof(Record) + 5 * 4 + 2 * 8 + sizeof(int4)) + rt + 8 * 256;
}

ts_status ts::render_views_hooked(ts_scene* const* scenes, const ts_camera* cams, int n_views, float* const* out_rgba,
                                  ts_saved** saved_out, void* stream, ReserveFn reserve, void* ctx) {
  if (!scenes || !cams || !out_rgba) return fail(TS_ERR_ARG, "ts_render_views: NULL argument");
  if (n_views < 1 || n_views > MAX_VIEWS) return fail(TS_ERR_ARG, "ts_render_views: n_views out of [1, 32]");
  const int device = scenes[0] ? scenes[0]->device : 0;
  for (int i = 0; i < n_views; ++i) {
    ts_status r = check_scene(scenes[i]);
    if (r != TS_OK) return r;
    if ((r = check_cam(&cams[i])) != TS_OK) return r;
    if (!out_rgba[i]) return fail(TS_ERR_ARG, "ts_render_views: NULL output");
    if (scenes[i]->device != device) return fail(TS_ERR_ARG, "ts_render_views: scenes on different devices");
    if (scenes[i]->tex_dtype != scenes[0]->tex_dtype)
      return fail(TS_ERR_ARG, "ts_render_views: views of one batch must share the atlas dtype");
    if (scenes[i]->sampler != scenes[0]->sampler)
      return fail(TS_ERR_ARG, "ts_render_views: views of one batch must share the texture sampler");
    if (scenes[i]->sampler == SMP_HW_ATLAS &&
        (!scenes[i]->a2d_tex[0] || scenes[i]->a2d_version != scenes[i]->tex_version || scenes[i]->a2d_n != scenes[i]->n))
      return fail(TS_ERR_STATE, "ts_render_views: hardware sampler selected but the 2-D atlas is missing or stale");
  }
  const int sampler = scenes[0]->sampler;
  bool indirect = false;
  for (int i = 0; i < n_views; ++i) {
    if (scenes[i]->sh && scenes[i]->sh_n != scenes[i]->n)
      return fail(TS_ERR_STATE, "ts_render_views: SH coefficients stale (re-upload after geometry)");
    indirect = indirect || (scenes[i]->sh != nullptr);
  }
  if (indirect && sampler != SMP_SOFTWARE)
    return fail(TS_ERR_STATE, "ts_render_views: indirect light (SH) needs the software sampler");
  for (int i = 1; i < n_views; ++i)
    if (scenes[i]->normal_xy != scenes[0]->normal_xy)
      return fail(TS_ERR_ARG, "ts_render_views: views of one batch must share the tangent-normal encoding");
  const int feat = (indirect ? FEAT_IND : 0) | (scenes[0]->normal_xy ? FEAT_N2 : 0);
  if (sampler != SMP_SOFTWARE && saved_out)
    return fail(TS_ERR_STATE, "ts_render_views: the hardware-atlas and flat samplers are inference-only (no saved state)");
  cudaStream_t st = (cudaStream_t)stream;
  TS_CUDA(cudaSetDevice(device));

  ViewTable vt;
  memset(&vt, 0, sizeof(vt));
  vt.n_views = n_views;
  long long tiles = 0, items = 0, pixels = 0;
  for (int i = 0; i < n_views; ++i) {
    const ts_camera& c = cams[i];
    const ts_scene* s = scenes[i];
    ViewDesc& V = vt.v[i];
    memcpy(V.R, c.R, sizeof(V.R));
    memcpy(V.t, c.t, sizeof(V.t));
    V.fx = c.fx; V.fy = c.fy; V.cx = c.cx; V.cy = c.cy;
    V.W = c.width; V.H = c.height;
    V.tiles_x = (c.width + TILE - 1) / TILE;
    V.tiles_y = (c.height + TILE - 1) / TILE;
    V.tile_off = (int)tiles;
    V.item_off = (int)items;
    V.pix_off = (int)pixels;
    V.n_splats = (int)s->n;
    V.means = s->means; V.quats = s->quats; V.scales = s->scales; V.opacity = s->opacity;
    V.texels = s->texels; V.T = s->T; V.tex_dtype = s->tex_dtype;
    V.tex_v8 = s->tex_dtype == DT_F32 && (reinterpret_cast<uintptr_t>(s->texels) & 31) == 0;
    V.atlas2d[0] = s->a2d_tex[0];
    V.atlas2d[1] = s->a2d_tex[1];
    V.chart = s->chart;
    V.sh = s->sh;
    V.sh_deg = s->sh ? s->sh_deg : 0;
    V.sh_stride = s->sh_stride;
    V.vis = s->sh ? c.visibility : nullptr;  // the indirect-light model only
    fill_env(s, V.env);
    V.rgba = reinterpret_cast<float4*>(out_rgba[i]);
    tiles += (long long)V.tiles_x * V.tiles_y;
    items += s->n;
    pixels += (long long)V.W * V.H;
  }
  if (items > INT32_MAX / 2 || tiles > INT32_MAX / 2 || pixels > INT32_MAX / 4)
    return fail(TS_ERR_CAPACITY, "ts_render_views: batch too large");
  vt.n_tiles = (int)tiles;
  vt.n_items = (int)items;
  const int n_items = vt.n_items;

  Scratch tmp(st);
  ts_saved* sv = nullptr;
  std::vector<void*> keep;  // buffers that move into the saved handle
  auto salloc = [&](void** p, size_t bytes) -> cudaError_t {
    if (saved_out) {
      cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 16, st);
      if (e == cudaSuccess) keep.push_back(*p);
      return e;
    }
    return tmp.alloc(p, bytes);
  };
  auto cleanup_keep = [&]() {
    for (void* p : keep) cudaFreeAsync(p, st);
    keep.clear();
  };
#define TS_CUDA_K(call)                                                                        \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      cleanup_keep();                                                                          \
      return fail(e_ == cudaErrorMemoryAllocation ? TS_ERR_OOM : TS_ERR_CUDA,                  \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                         \
    }                                                                                          \
  } while (0)

  // ---- per-item preprocess --------------------------------------------------
  Record* rec = nullptr;
  uint32_t *counts = nullptr, *ids0 = nullptr, *ids1 = nullptr, *cs = nullptr, *offs = nullptr, *dbits = nullptr;
  uint64_t *dk0 = nullptr, *dk1 = nullptr;
  int4* rects = nullptr;
  const size_t ni = (size_t)std::max(n_items, 1);
  TS_CUDA_K(salloc((void**)&rec, ni * sizeof(Record)));
  TS_CUDA_K(tmp.alloc((void**)&counts, ni * 4));
  TS_CUDA_K(tmp.alloc((void**)&ids0, ni * 4));
  TS_CUDA_K(tmp.alloc((void**)&ids1, ni * 4));
  TS_CUDA_K(tmp.alloc((void**)&cs, ni * 4));
  TS_CUDA_K(tmp.alloc((void**)&offs, ni * 4));
  TS_CUDA_K(tmp.alloc((void**)&dk0, ni * 8));
  TS_CUDA_K(tmp.alloc((void**)&dk1, ni * 8));
  TS_CUDA_K(tmp.alloc((void**)&rects, ni * sizeof(int4)));
  if (saved_out) TS_CUDA_K(salloc((void**)&dbits, ni * 4));
  void* rtemp = nullptr;
  size_t rt_bytes = std::max(radix_temp_bytes(n_items, 8), scan_temp_bytes(n_items));
  TS_CUDA_K(tmp.alloc(&rtemp, rt_bytes));

  {
    ProfScope p(st, "preprocess");
    launch_preprocess(vt, rec, counts, dk0, ids0, rects, st);
    if (dbits) launch_depth_bits(dk0, dbits, n_items, st);
  }
  const int view_bits = bits_for(n_views);
  int which = 0;
  {
    ProfScope p(st, "sort_splats");
    which = radix_sort_u64(dk0, ids0, dk1, ids1, n_items, 0, 32 + view_bits, rtemp, st);
  }
  uint32_t* order = which ? ids1 : ids0;
  {
    ProfScope p(st, "scan_counts");
    launch_gather_counts(order, counts, cs, n_items, st);
    launch_exclusive_scan(cs, offs, n_items, rtemp, st);
  }
  // a batch whose pair count could pass 2^31 (n x tiles bound) also sums the
  // counts in 64 bits: the 32-bit scan above would wrap
  unsigned long long* d_total = nullptr;
  {
    long long bound = 0;
    for (int i = 0; i < n_views; ++i) bound += (long long)vt.v[i].n_splats * vt.v[i].tiles_x * vt.v[i].tiles_y;
    if (bound > INT32_MAX / 2) {
      TS_CUDA_K(tmp.alloc((void**)&d_total, sizeof(unsigned long long)));
      launch_sum_counts(cs, n_items, d_total, st);
    }
  }
  TS_CHECK_LAUNCH();

  // total pair count -> host (one synchronisation per batch)
  struct HostTail {
    uint32_t tail[2];
    unsigned long long total;
    int sort_err[2];
  };
  int* d_sort_err = sort_error_flag(device);
  vt.sort_err = d_sort_err;
  static thread_local HostTail* h_tail = nullptr;
  if (!h_tail) TS_CUDA_K(cudaHostAlloc((void**)&h_tail, sizeof(HostTail), cudaHostAllocPortable));
  h_tail->tail[0] = h_tail->tail[1] = 0;
  h_tail->total = 0;
  h_tail->sort_err[0] = h_tail->sort_err[1] = 0;
  if (d_sort_err) TS_CUDA_K(cudaMemcpyAsync(h_tail->sort_err, d_sort_err, 8, cudaMemcpyDeviceToHost, st));
  if (n_items > 0) {
    TS_CUDA_K(cudaMemcpyAsync(&h_tail->tail[0], offs + (n_items - 1), 4, cudaMemcpyDeviceToHost, st));
    TS_CUDA_K(cudaMemcpyAsync(&h_tail->tail[1], cs + (n_items - 1), 4, cudaMemcpyDeviceToHost, st));
    if (d_total) TS_CUDA_K(cudaMemcpyAsync(&h_tail->total, d_total, 8, cudaMemcpyDeviceToHost, st));
  }
  TS_CUDA_K(cudaStreamSynchronize(st));
  if (h_tail->sort_err[SORT_FLAG_LISTS]) {  // the depth sort's bounded wait ran out (this batch)
    cudaMemsetAsync(d_sort_err, 0, 2 * sizeof(int), st);
    cleanup_keep();
    return fail(TS_ERR_TIMEOUT, "ts_render_views: a radix-sort look-back wait ran out");
  }
  // an earlier call's launch-order sort ran out: its rasteriser took the
  // tiles in tile order (same result); the word is cleared for this call
  if (h_tail->sort_err[SORT_FLAG_ORDER]) TS_CUDA_K(cudaMemsetAsync(d_sort_err + SORT_FLAG_ORDER, 0, sizeof(int), st));
  const long long K = (long long)h_tail->tail[0] + h_tail->tail[1];
  if (K > INT32_MAX / 2 || (d_total && h_tail->total > (unsigned long long)(INT32_MAX / 2))) {
    cleanup_keep();
    return fail(TS_ERR_CAPACITY, "ts_render_views: too many (tile, splat) pairs");
  }
  if (reserve) {  // the caller admits the rest of the call's memory now that K is known
    size_t rest = (size_t)std::max<long long>(K, 1) * 16 + (size_t)vt.n_tiles * (8 + 16) +
                  std::max(radix_temp_bytes((int)K, 4), radix_temp_bytes(vt.n_tiles, 4)) + 8 * 256;
    if (saved_out) rest += (size_t)pixels * (32 + 4 + 4 + 4 + 4 + (indirect ? 16 : 0));
    const ts_status r = reserve(ctx, rest, K);
    if (r != TS_OK) {
      cleanup_keep();
      return r;
    }
  }

  // ---- pairs: emit in depth order, stable sort by tile --------------------------
  uint32_t *tk0 = nullptr, *tk1 = nullptr, *pi0 = nullptr, *pi1 = nullptr;
  uint2* ranges = nullptr;
  const size_t nk = (size_t)std::max<long long>(K, 1);
  TS_CUDA_K(salloc((void**)&tk0, nk * 4));
  TS_CUDA_K(salloc((void**)&pi0, nk * 4));
  TS_CUDA_K(salloc((void**)&tk1, nk * 4));
  TS_CUDA_K(salloc((void**)&pi1, nk * 4));
  TS_CUDA_K(salloc((void**)&ranges, (size_t)vt.n_tiles * sizeof(uint2)));
  uint32_t* obuf = nullptr;  // tile launch order: keys and ids, twice
  TS_CUDA_K(salloc((void**)&obuf, (size_t)vt.n_tiles * 4 * sizeof(uint32_t)));
  void* rtemp2 = nullptr;
  TS_CUDA_K(tmp.alloc(&rtemp2, std::max(radix_temp_bytes((int)K, 4), radix_temp_bytes(vt.n_tiles, 4))));
  {
    ProfScope p(st, "emit_pairs");
    launch_emit_pairs(vt, order, offs, cs, rects, tk0, pi0, n_items, st);
  }
  int w2 = 0;
  {
    ProfScope p(st, "sort_pairs");
    w2 = radix_sort_u32(tk0, pi0, tk1, pi1, (int)K, 0, std::max(1, bits_for(vt.n_tiles)), rtemp2, st, -1);
  }
  uint32_t* tkeys = w2 ? tk1 : tk0;
  uint32_t* pitems = w2 ? pi1 : pi0;
  {
    ProfScope p(st, "tile_ranges");
    TS_CUDA_K(cudaMemsetAsync(ranges, 0, (size_t)vt.n_tiles * sizeof(uint2), st));
    launch_tile_ranges(tkeys, (int)K, vt.n_tiles, ranges, st);
    vt.tile_order = launch_tile_order(ranges, vt.n_tiles, obuf, rtemp2, st);
  }
  TS_CHECK_LAUNCH();

  // ---- per-pixel state for the backward ------------------------------------------
  if (saved_out) {
    for (int i = 0; i < n_views; ++i) {
      ViewDesc& V = vt.v[i];
      const size_t np = (size_t)V.W * V.H;
      TS_CUDA_K(salloc((void**)&V.gbuf, np * 2 * sizeof(float4)));
      TS_CUDA_K(salloc((void**)&V.trans, np * sizeof(float)));
      TS_CUDA_K(salloc((void**)&V.acc, np * sizeof(float)));
      TS_CUDA_K(salloc((void**)&V.zsum, np * sizeof(float)));
      if (indirect) TS_CUDA_K(salloc((void**)&V.gind, np * sizeof(float4)));
      TS_CUDA_K(salloc((void**)&V.last, np * sizeof(int)));
    }
  }
  {
    ProfScope p(st, "raster_fwd");
    launch_raster_fwd(vt, rec, pitems, ranges, scenes[0]->tex_dtype, saved_out != nullptr, nullptr, sampler, feat, st);
  }
  TS_CHECK_LAUNCH();

  if (saved_out) {
    sv = new (std::nothrow) ts_saved();
    if (!sv) {
      cleanup_keep();
      return fail(TS_ERR_OOM, "ts_render_views: host allocation failed");
    }
    sv->device = device;
    sv->stream = st;
    sv->vt = vt;
    sv->indirect = indirect;
    sv->feat = feat;
    sv->scenes.assign(scenes, scenes + n_views);
    for (int i = 0; i < n_views; ++i) sv->gens.push_back(scenes[i]->gen);
    sv->rec = rec;
    sv->pair_items = pitems;
    sv->tile_keys = tkeys;
    sv->ranges = ranges;
    sv->depth_bits = dbits;
    sv->K = K;
    sv->bufs = keep;
    *saved_out = sv;
  }
  return TS_OK;
#undef TS_CUDA_K
}

extern "C" {

ts_status ts_render_views(ts_scene* const* scenes, const ts_camera* cams, int n_views, float* const* out_rgba,
                          ts_saved** saved_out, void* stream) {
  return ts::render_views_hooked(scenes, cams, n_views, out_rgba, saved_out, stream, nullptr, nullptr);
}

ts_status ts_render(ts_scene* scene, const ts_camera* cam, float* out_rgba, ts_saved** saved, void* stream) {
  ts_scene* sc[1] = {scene};
  float* outs[1] = {out_rgba};
  return ts_render_views(sc, cam, 1, outs, saved, stream);
}

ts_status ts_release_saved(ts_saved* sv) {
  if (!sv) return TS_OK;
  cudaSetDevice(sv->device);
  for (void* p : sv->bufs) cudaFreeAsync(p, sv->stream);
  delete sv;
  return TS_OK;
}

ts_status ts_render_backward(const ts_saved* sv, const float* const* dL_drgba, const ts_grads* grads, void* stream) {
  if (!sv || !dL_drgba || !grads) return fail(TS_ERR_ARG, "ts_render_backward: NULL argument");
  if (!scenes_unchanged(sv))
    return fail(TS_ERR_STATE, "ts_render_backward: a scene was re-uploaded since the forward (render again)");
  const ts_scene* s = sv->scenes[0];
  for (ts_scene* o : sv->scenes)
    if (o != s) return fail(TS_ERR_ARG, "ts_render_backward: views of one backward must share one scene");
  cudaStream_t st = (cudaStream_t)stream;
  TS_CUDA(cudaSetDevice(sv->device));
  ViewTable vt = sv->vt;
  for (int i = 0; i < vt.n_views; ++i) {
    if (!dL_drgba[i]) return fail(TS_ERR_ARG, "ts_render_backward: NULL dL/drgba");
    vt.v[i].dl = reinterpret_cast<const float4*>(dL_drgba[i]);
  }
  GradTable g;
  memset(&g, 0, sizeof(g));
  g.means = grads->means;
  g.quats = grads->quats;
  g.scales = grads->scales;
  g.opacity = grads->opacity;
  g.texels = grads->texels;
  g.irr = grads->irr;
  g.sh = grads->sh;
  if (grads->spec) {
    for (int l = 0; l < s->levels; ++l) g.spec[l] = grads->spec + s->spec_off[l];
  }
  Scratch tmp(st);
  double* g_items = nullptr;
  float4* gxa = nullptr;
  long long n_pix = 0;
  for (int i = 0; i < vt.n_views; ++i) n_pix += (long long)vt.v[i].W * vt.v[i].H;
  TS_CUDA(tmp.alloc((void**)&g_items, (size_t)std::max(vt.n_items, 1) * kRecGradStride * sizeof(double)));
  TS_CUDA(tmp.alloc((void**)&gxa, (size_t)std::max(n_pix, 1ll) * 3 * sizeof(float4)));
  TS_CUDA(cudaMemsetAsync(g_items, 0, (size_t)std::max(vt.n_items, 1) * kRecGradStride * sizeof(double), st));
  if (sv->indirect) {  // per-pixel dL/dX_ind between the shading and raster adjoints
    for (int i = 0; i < vt.n_views; ++i)
      TS_CUDA(tmp.alloc((void**)&vt.v[i].gxind, (size_t)vt.v[i].W * vt.v[i].H * sizeof(float4)));
  }
  {
    ProfScope p(st, "shade_bwd");
    launch_shade_bwd(vt, gxa, g, st);
  }
  {
    ProfScope p(st, "raster_bwd");
    // tiles by the entries the backward walks, longest first
    uint32_t* obuf = nullptr;
    void* otemp = nullptr;
    TS_CUDA(tmp.alloc((void**)&obuf, (size_t)std::max(vt.n_tiles, 1) * 4 * sizeof(uint32_t)));
    TS_CUDA(tmp.alloc(&otemp, radix_temp_bytes(vt.n_tiles, 4)));
    vt.tile_order = launch_tile_order_walk(vt, sv->ranges, obuf, otemp, st);
    launch_raster_bwd(vt, sv->rec, sv->pair_items, sv->ranges, s->tex_dtype, gxa, g_items, g, sv->feat, st);
  }
  {
    ProfScope p(st, "preprocess_bwd");
    launch_preprocess_bwd(vt, g_items, g, st);
  }
  TS_CHECK_LAUNCH();
  return TS_OK;
}

ts_status ts_saved_sizes(const ts_saved* sv, int64_t* n_pairs, int64_t* n_tiles) {
  if (!sv) return fail(TS_ERR_ARG, "ts_saved_sizes: NULL saved");
  if (n_pairs) *n_pairs = sv->K;
  if (n_tiles) *n_tiles = sv->vt.n_tiles;
  return TS_OK;
}

ts_status ts_saved_copy_lists(const ts_saved* sv, uint32_t* item_ids, uint32_t* tile_ranges, uint32_t* depth_bits,
                              void* stream) {
  if (!sv) return fail(TS_ERR_ARG, "ts_saved_copy_lists: NULL saved");
  cudaStream_t st = (cudaStream_t)stream;
  TS_CUDA(cudaSetDevice(sv->device));
  if (item_ids && sv->K > 0)
    TS_CUDA(cudaMemcpyAsync(item_ids, sv->pair_items, (size_t)sv->K * 4, cudaMemcpyDeviceToDevice, st));
  if (tile_ranges)
    TS_CUDA(cudaMemcpyAsync(tile_ranges, sv->ranges, (size_t)sv->vt.n_tiles * 8, cudaMemcpyDeviceToDevice, st));
  if (depth_bits && sv->vt.n_items > 0)
    TS_CUDA(cudaMemcpyAsync(depth_bits, sv->depth_bits, (size_t)sv->vt.n_items * 4, cudaMemcpyDeviceToDevice, st));
  return TS_OK;
}

ts_status ts_saved_copy_pixels(const ts_saved* sv, int view, float* gbuf, float* trans, int32_t* last, void* stream) {
  if (!sv) return fail(TS_ERR_ARG, "ts_saved_copy_pixels: NULL saved");
  if (view < 0 || view >= sv->vt.n_views) return fail(TS_ERR_ARG, "ts_saved_copy_pixels: bad view");
  cudaStream_t st = (cudaStream_t)stream;
  TS_CUDA(cudaSetDevice(sv->device));
  const ViewDesc& V = sv->vt.v[view];
  const size_t np = (size_t)V.W * V.H;
  if (gbuf) TS_CUDA(cudaMemcpyAsync(gbuf, V.gbuf, np * 32, cudaMemcpyDeviceToDevice, st));
  if (trans) TS_CUDA(cudaMemcpyAsync(trans, V.trans, np * 4, cudaMemcpyDeviceToDevice, st));
  if (last) TS_CUDA(cudaMemcpyAsync(last, V.last, np * 4, cudaMemcpyDeviceToDevice, st));
  return TS_OK;
}

ts_status ts_saved_copy_depth(const ts_saved* sv, int view, float* zsum, float* acc, void* stream) {
  if (!sv) return fail(TS_ERR_ARG, "ts_saved_copy_depth: NULL saved");
  if (view < 0 || view >= sv->vt.n_views) return fail(TS_ERR_ARG, "ts_saved_copy_depth: bad view");
  cudaStream_t st = (cudaStream_t)stream;
  TS_CUDA(cudaSetDevice(sv->device));
  const ViewDesc& V = sv->vt.v[view];
  const size_t np = (size_t)V.W * V.H;
  if (zsum) TS_CUDA(cudaMemcpyAsync(zsum, V.zsum, np * 4, cudaMemcpyDeviceToDevice, st));
  if (acc) TS_CUDA(cudaMemcpyAsync(acc, V.acc, np * 4, cudaMemcpyDeviceToDevice, st));
  return TS_OK;
}

ts_status ts_normal_loss(ts_saved* sv, int view, float weight, float* loss, void* stream) {
  if (!sv || !loss) return fail(TS_ERR_ARG, "ts_normal_loss: NULL argument");
  if (view < 0 || view >= sv->vt.n_views) return fail(TS_ERR_ARG, "ts_normal_loss: bad view");
  if (!(weight >= 0.f)) return fail(TS_ERR_ARG, "ts_normal_loss: weight must be >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  TS_CUDA(cudaSetDevice(sv->device));
  ViewDesc& V = sv->vt.v[view];
  const size_t np = (size_t)V.W * V.H;
  if (!V.gnorm) {  // per-view gradient buffers, owned by the saved state
    void* a = nullptr;
    void* b = nullptr;
    TS_CUDA(cudaMallocAsync(&a, np * sizeof(float4), sv->stream));
    TS_CUDA(cudaMallocAsync(&b, np * sizeof(float), sv->stream));
    sv->bufs.push_back(a);
    sv->bufs.push_back(b);
    V.gnorm = reinterpret_cast<const float4*>(a);
    V.gzsum = reinterpret_cast<const float*>(b);
    if (st != sv->stream) TS_CUDA(cudaStreamSynchronize(sv->stream));
  }
  void* temp = nullptr;
  TS_CUDA(cudaMallocAsync(&temp, normal_loss_temp_bytes(V.W, V.H), st));
  {
    ProfScope p(st, "normal_loss");
    launch_normal_loss(V, weight, loss, const_cast<float4*>(V.gnorm), const_cast<float*>(V.gzsum), temp, st);
  }
  const cudaError_t e = cudaGetLastError();
  cudaFreeAsync(temp, st);
  if (e != cudaSuccess) return fail(TS_ERR_CUDA, std::string("ts_normal_loss: ") + cudaGetErrorString(e));
  return TS_OK;
}

ts_status ts_saved_frag_stats(const ts_saved* sv, ts_frag_stats* out, void* stream) {
  if (!sv || !out) return fail(TS_ERR_ARG, "ts_saved_frag_stats: NULL argument");
  if (!scenes_unchanged(sv))
    return fail(TS_ERR_STATE, "ts_saved_frag_stats: a scene was re-uploaded since the forward (render again)");
  cudaStream_t st = (cudaStream_t)stream;
  TS_CUDA(cudaSetDevice(sv->device));
  ViewTable vt = sv->vt;
  Scratch tmp(st);
  for (int i = 0; i < vt.n_views; ++i) {
    ViewDesc& V = vt.v[i];
    TS_CUDA(tmp.alloc((void**)&V.rgba, (size_t)V.W * V.H * sizeof(float4)));
  }
  unsigned long long* d = nullptr;
  TS_CUDA(tmp.alloc((void**)&d, 4 * sizeof(unsigned long long)));
  TS_CUDA(cudaMemsetAsync(d, 0, 4 * sizeof(unsigned long long), st));
  // texel bitmap: one bit per texel of each list item's chart
  int t2max = 1;
  for (int i = 0; i < vt.n_views; ++i) t2max = std::max(t2max, vt.v[i].T * vt.v[i].T);
  const int wpi = (t2max + 31) / 32;
  const size_t bm_bytes = (size_t)std::max<long long>(vt.n_items, 1) * wpi * 4;
  uint32_t* bm = nullptr;
  TS_CUDA(tmp.alloc((void**)&bm, bm_bytes));
  TS_CUDA(cudaMemsetAsync(bm, 0, bm_bytes, st));
  const FragCounters fc{d, bm, wpi};
  launch_raster_fwd(vt, sv->rec, sv->pair_items, sv->ranges, sv->scenes[0]->tex_dtype, false, &fc, SMP_SOFTWARE, 0,
                    st);
  TS_CHECK_LAUNCH();
  launch_touch_counts(bm, vt.n_items, wpi, d, st);
  TS_CHECK_LAUNCH();
  unsigned long long h[4] = {0, 0, 0, 0};
  TS_CUDA(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
  // visible splats: items with a finite depth
  uint32_t* db = sv->depth_bits;
  std::vector<uint32_t> hb((size_t)vt.n_items);
  if (db && vt.n_items > 0)
    TS_CUDA(cudaMemcpyAsync(hb.data(), db, (size_t)vt.n_items * 4, cudaMemcpyDeviceToHost, st));
  TS_CUDA(cudaStreamSynchronize(st));
  out->n_pairs = sv->K;
  out->n_evaluated = (int64_t)h[0];
  out->n_blended = (int64_t)h[1];
  out->n_texels_read = (int64_t)h[2];
  out->n_items_blended = (int64_t)h[3];
  int64_t vis = 0;
  for (uint32_t b : hb) vis += (b != 0xffffffffu);
  out->n_visible = vis;
  return TS_OK;
}

ts_status ts_upload_indirect(ts_scene* s, int degree, const float* coeffs, int src_on_device, void* stream) {
  if (!s) return fail(TS_ERR_ARG, "ts_upload_indirect: scene is NULL");
  if (degree < -1 || degree > 2) return fail(TS_ERR_ARG, "ts_upload_indirect: degree must be -1, 0, 1 or 2");
  cudaStream_t st = (cudaStream_t)stream;
  TS_CUDA(cudaSetDevice(s->device));
  if (degree >= 0 && s->sh && s->sh_deg == degree && s->sh_n == s->n) {
    // same degree and splat count: overwrite in place, stream-ordered (training updates)
    if (s->n > 0 && !coeffs) return fail(TS_ERR_ARG, "ts_upload_indirect: coeffs is NULL");
    const int K = (degree + 1) * (degree + 1);
    if (s->n > 0)
      TS_CUDA(cudaMemcpy2DAsync(s->sh, s->sh_stride * sizeof(float), coeffs, 3 * K * sizeof(float),
                                3 * K * sizeof(float), (size_t)s->n,
                                src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    if (!src_on_device) TS_CUDA(cudaStreamSynchronize(st));
    return TS_OK;
  }
  TS_CUDA(cudaStreamSynchronize(st));
  if (s->sh) cudaFree(s->sh);
  s->gen += 1;
  s->sh = nullptr;
  s->sh_deg = -1;
  s->sh_stride = 0;
  s->sh_n = -1;
  if (degree < 0) return TS_OK;
  if (!s->means) return fail(TS_ERR_STATE, "ts_upload_indirect: geometry not uploaded");
  if (s->n > 0 && !coeffs) return fail(TS_ERR_ARG, "ts_upload_indirect: coeffs is NULL");
  const int K = (degree + 1) * (degree + 1);
  const int stride = (3 * K + 3) & ~3;
  const size_t n = (size_t)std::max<int64_t>(s->n, 1);
  TS_CUDA(dev_malloc((void**)&s->sh, n * stride * sizeof(float)));
  TS_CUDA(cudaMemsetAsync(s->sh, 0, n * stride * sizeof(float), st));
  if (s->n > 0)
    TS_CUDA(cudaMemcpy2DAsync(s->sh, stride * sizeof(float), coeffs, 3 * K * sizeof(float), 3 * K * sizeof(float),
                              (size_t)s->n, src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  TS_CUDA(cudaStreamSynchronize(st));
  s->sh_deg = degree;
  s->sh_stride = stride;
  s->sh_n = s->n;
  return TS_OK;
}

ts_status ts_scene_build_atlas2d(ts_scene* s, ts_dtype store, int packing, void* stream) {
  if (!s) return fail(TS_ERR_ARG, "ts_scene_build_atlas2d: scene is NULL");
  if (packing != TS_PACK_SPLAT_ID && packing != TS_PACK_MORTON)
    return fail(TS_ERR_ARG, "ts_scene_build_atlas2d: unknown packing");
  if (store != TS_F32 && store != TS_F16) return fail(TS_ERR_ARG, "ts_scene_build_atlas2d: store must be TS_F32 or TS_F16");
  if (!s->texels || s->tex_n != s->n) return fail(TS_ERR_STATE, "ts_scene_build_atlas2d: atlas missing or stale");
  cudaStream_t st = (cudaStream_t)stream;
  TS_CUDA(cudaSetDevice(s->device));
  TS_CUDA(cudaStreamSynchronize(st));
  free_atlas2d(s);
  const int T = s->T;
  const long long n = std::max<long long>(s->n, 1);
  int max_w = 0, max_h = 0;
  TS_CUDA(cudaDeviceGetAttribute(&max_w, cudaDevAttrMaxSurface2DWidth, s->device));
  TS_CUDA(cudaDeviceGetAttribute(&max_h, cudaDevAttrMaxSurface2DHeight, s->device));
  // near-square atlas (power-of-two width): small texel coordinates keep FP32
  // sub-texel precision well below the filter's 1/256 weight step
  long long w = T;
  while (w * 2 <= max_w && w * w < n * T * T) w *= 2;
  long long charts_x = w / T, rows = (n + charts_x - 1) / charts_x;
  while (rows * T > max_h && w * 2 <= max_w) {
    w *= 2;
    charts_x = w / T;
    rows = (n + charts_x - 1) / charts_x;
  }
  if (rows * T > max_h) return fail(TS_ERR_CAPACITY, "ts_scene_build_atlas2d: too many charts for one 2-D texture");
  const int W = (int)w, H = (int)(rows * T);
  const cudaChannelFormatDesc desc =
      store == TS_F32 ? cudaCreateChannelDesc<float4>() : cudaCreateChannelDescHalf4();
  cudaSurfaceObject_t surf[2] = {0, 0};
  ts_status r = TS_OK;
  for (int i = 0; i < 2 && r == TS_OK; ++i) {
    if (cudaMallocArray(&s->a2d[i], &desc, W, H, cudaArraySurfaceLoadStore) != cudaSuccess) {
      r = fail(TS_ERR_OOM, "ts_scene_build_atlas2d: array allocation failed");
      break;
    }
    cudaResourceDesc res;
    memset(&res, 0, sizeof(res));
    res.resType = cudaResourceTypeArray;
    res.res.array.array = s->a2d[i];
    if (cudaCreateSurfaceObject(&surf[i], &res) != cudaSuccess) {
      r = fail(TS_ERR_CUDA, "ts_scene_build_atlas2d: surface creation failed");
      break;
    }
    cudaTextureDesc td;
    memset(&td, 0, sizeof(td));
    td.addressMode[0] = td.addressMode[1] = cudaAddressModeClamp;
    td.filterMode = cudaFilterModeLinear;
    td.readMode = cudaReadModeElementType;
    td.normalizedCoords = 0;
    if (cudaCreateTextureObject(&s->a2d_tex[i], &res, &td, nullptr) != cudaSuccess)
      r = fail(TS_ERR_CUDA, "ts_scene_build_atlas2d: texture creation failed");
  }
  if (r == TS_OK && cudaMalloc(&s->chart, (size_t)n * sizeof(uint2)) != cudaSuccess)
    r = fail(TS_ERR_OOM, "ts_scene_build_atlas2d: indirection buffer allocation failed");
  // chart order: splat id (the paper's packing) or the Morton order of the
  // splat centres, so that splats near each other in space get neighbouring
  // charts (the locality-aware packing the paper leaves to future work)
  uint32_t* chart_of = nullptr;
  void* mtemp = nullptr;
  if (r == TS_OK && s->n > 0 && packing == TS_PACK_MORTON) {
    const size_t nn = (size_t)s->n;
    const size_t rt = radix_temp_bytes((int)s->n, 4);
    const size_t bytes = 256 + 5 * ((nn * 4 + 255) & ~size_t(255)) + rt;
    if (cudaMalloc(&mtemp, bytes) != cudaSuccess) {
      r = fail(TS_ERR_OOM, "ts_scene_build_atlas2d: scratch allocation failed");
    } else {
      char* b = reinterpret_cast<char*>(mtemp);
      const size_t seg = (nn * 4 + 255) & ~size_t(255);
      uint32_t* bbox = reinterpret_cast<uint32_t*>(b);
      uint32_t* k0 = reinterpret_cast<uint32_t*>(b + 256);
      uint32_t* v0 = reinterpret_cast<uint32_t*>(b + 256 + seg);
      uint32_t* k1 = reinterpret_cast<uint32_t*>(b + 256 + 2 * seg);
      uint32_t* v1 = reinterpret_cast<uint32_t*>(b + 256 + 3 * seg);
      chart_of = reinterpret_cast<uint32_t*>(b + 256 + 4 * seg);
      void* rtemp = b + 256 + 5 * seg;
      launch_morton_order(s->means, s->n, bbox, k0, v0, st);
      const int w = radix_sort_u32(k0, v0, k1, v1, (int)s->n, 0, 30, rtemp, st, -1);
      launch_chart_of(w ? v1 : v0, s->n, chart_of, st);
    }
  }
  if (r == TS_OK && s->n > 0) {
    launch_pack_atlas2d(s->texels, s->tex_dtype, s->n, T, (int)charts_x, surf[0], surf[1], s->chart, chart_of,
                        store == TS_F16 ? 1 : 0, st);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
      r = fail(TS_ERR_CUDA, "ts_scene_build_atlas2d: packing failed");
  }
  if (mtemp) {
    cudaStreamSynchronize(st);
    cudaFree(mtemp);
  }
  for (int i = 0; i < 2; ++i)
    if (surf[i]) cudaDestroySurfaceObject(surf[i]);
  if (r != TS_OK) {
    free_atlas2d(s);
    return r;
  }
  s->a2d_version = s->tex_version;
  s->a2d_n = s->n;
  return TS_OK;
}

ts_status ts_scene_set_sampler(ts_scene* s, int sampler) {
  if (!s) return fail(TS_ERR_ARG, "ts_scene_set_sampler: scene is NULL");
  if (sampler != SMP_SOFTWARE && sampler != SMP_HW_ATLAS && sampler != SMP_FLAT)
    return fail(TS_ERR_ARG, "ts_scene_set_sampler: unknown sampler");
  s->sampler = sampler;
  return TS_OK;
}

ts_status ts_scene_set_normal_encoding(ts_scene* s, int encoding) {
  if (!s) return fail(TS_ERR_ARG, "ts_scene_set_normal_encoding: scene is NULL");
  if (encoding != TS_NORMAL_XYZ && encoding != TS_NORMAL_XY)
    return fail(TS_ERR_ARG, "ts_scene_set_normal_encoding: unknown encoding");
  s->normal_xy = encoding == TS_NORMAL_XY;
  return TS_OK;
}

ts_status ts_image_loss(const float* rgba, const float* target, int width, int height, float lambda_dssim,
                        float* loss, float* grad, void* stream) {
  if (!rgba || !target || !loss || !grad) return fail(TS_ERR_ARG, "ts_image_loss: NULL argument");
  if (width < 1 || height < 1 || (long long)width * height > (1ll << 28))
    return fail(TS_ERR_ARG, "ts_image_loss: image size out of range");
  if (!(lambda_dssim >= 0.f && lambda_dssim <= 1.f)) return fail(TS_ERR_ARG, "ts_image_loss: lambda not in [0, 1]");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  TS_CUDA(cudaGetDevice(&dev));
  if (set_gauss_window(dev) != 0) return fail(TS_ERR_CUDA, "ts_image_loss: window upload failed");
  void* temp = nullptr;
  TS_CUDA(cudaMallocAsync(&temp, image_loss_temp_bytes(width, height), st));
  {
    ProfScope p(st, "image_loss");
    launch_image_loss(reinterpret_cast<const float4*>(rgba), reinterpret_cast<const float4*>(target), width, height,
                      lambda_dssim, loss, reinterpret_cast<float4*>(grad), temp, st);
  }
  const cudaError_t e = cudaGetLastError();
  cudaFreeAsync(temp, st);
  if (e != cudaSuccess) return fail(TS_ERR_CUDA, std::string("ts_image_loss: ") + cudaGetErrorString(e));
  return TS_OK;
}

ts_status ts_scene_texels(ts_scene* s, void** texels, int* T, int* dtype) {
  if (!s) return fail(TS_ERR_ARG, "ts_scene_texels: scene is NULL");
  if (!s->texels) return fail(TS_ERR_STATE, "ts_scene_texels: atlas not uploaded");
  if (texels) *texels = s->texels;
  if (T) *T = s->T;
  if (dtype) *dtype = s->tex_dtype;
  return TS_OK;
}

ts_status ts_scene_envmap(ts_scene* s, void** spec, void** irr, int* dtype) {
  if (!s) return fail(TS_ERR_ARG, "ts_scene_envmap: scene is NULL");
  if (!s->spec || !s->irr) return fail(TS_ERR_STATE, "ts_scene_envmap: environment not uploaded");
  if (spec) *spec = s->spec;
  if (irr) *irr = s->irr;
  if (dtype) *dtype = s->cube_dtype;
  return TS_OK;
}

ts_status ts_scene_set_geometry(ts_scene* s, const float* means, const float* quats, const float* scales,
                                const float* opacity, void* stream) {
  if (!s || !means || !quats || !scales || !opacity) return fail(TS_ERR_ARG, "ts_scene_set_geometry: NULL argument");
  if (!s->means) return fail(TS_ERR_STATE, "ts_scene_set_geometry: geometry not uploaded");
  cudaStream_t st = (cudaStream_t)stream;
  TS_CUDA(cudaSetDevice(s->device));
  const size_t n = (size_t)s->n;
  if (n == 0) return TS_OK;
  launch_pad4(means, 3, s->means, (long long)n, st);
  TS_CHECK_LAUNCH();
  TS_CUDA(cudaMemcpyAsync(s->quats, quats, n * 16, cudaMemcpyDeviceToDevice, st));
  TS_CUDA(cudaMemcpyAsync(s->scales, scales, n * 8, cudaMemcpyDeviceToDevice, st));
  TS_CUDA(cudaMemcpyAsync(s->opacity, opacity, n * 4, cudaMemcpyDeviceToDevice, st));
  return TS_OK;
}

ts_status ts_adam_update(float* param, float* grad, float* m, float* v, int64_t n, const ts_adam* hp, void* shadow,
                         ts_dtype shadow_dtype, int zero_grad, void* stream) {
  if (!param || !grad || !m || !v || !hp || n < 0) return fail(TS_ERR_ARG, "ts_adam_update: bad argument");
  const uintptr_t al = reinterpret_cast<uintptr_t>(param) | reinterpret_cast<uintptr_t>(grad) |
                       reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(v);
  if (al & 15) return fail(TS_ERR_ARG, "ts_adam_update: arrays must be 16-byte aligned");
  if (shadow && (reinterpret_cast<uintptr_t>(shadow) & 15)) return fail(TS_ERR_ARG, "ts_adam_update: shadow alignment");
  if (hp->step < 1 || !(hp->beta1 >= 0.f && hp->beta1 < 1.f) || !(hp->beta2 >= 0.f && hp->beta2 < 1.f))
    return fail(TS_ERR_ARG, "ts_adam_update: bad hyper-parameters");
  ProfScope p((cudaStream_t)stream, "adam");
  launch_adam(param, grad, m, v, n, hp->lr, hp->beta1, hp->beta2, hp->eps, hp->step, shadow, (int)shadow_dtype,
              zero_grad, (cudaStream_t)stream);
  TS_CHECK_LAUNCH();
  return TS_OK;
}

ts_status ts_scene_info(const ts_scene* s, int64_t* n, int* T, int* dtype) {
  if (!s) return fail(TS_ERR_ARG, "ts_scene_info: scene is NULL");
  if (!s->means || !s->texels) return fail(TS_ERR_STATE, "ts_scene_info: geometry or atlas missing");
  if (n) *n = s->n;
  if (T) *T = s->T;
  if (dtype) *dtype = s->tex_dtype;
  return TS_OK;
}

ts_status ts_debug_fail_alloc(int64_t after) {
  if (after < -1) return fail(TS_ERR_ARG, "ts_debug_fail_alloc: after must be >= -1");
  g_fail_alloc.store(after);
  return TS_OK;
}

ts_status ts_selftest_sort_wait(int device, void* stream) {
  TS_CUDA(cudaSetDevice(device));
  const int r = sort_wait_selftest((cudaStream_t)stream);
  if (r < 0) return fail(TS_ERR_CUDA, "ts_selftest_sort_wait: CUDA error");
  if (r == 0) return fail(TS_ERR_STATE, "ts_selftest_sort_wait: the wait did not report running out");
  return fail(TS_ERR_TIMEOUT, "ts_selftest_sort_wait: the bounded look-back wait ran out and was reported");
}

ts_status ts_activate(int64_t n, const float* log_scales, const float* logit_opacity, float* scales, float* opacity,
                      void* stream) {
  if (n < 0 || (n > 0 && (!log_scales || !logit_opacity || !scales || !opacity)))
    return fail(TS_ERR_ARG, "ts_activate: bad argument");
  launch_activate(log_scales, logit_opacity, n, scales, opacity, (cudaStream_t)stream);
  TS_CHECK_LAUNCH();
  return TS_OK;
}

ts_status ts_activate_backward(int64_t n, const float* scales, const float* opacity, const float* g_scales,
                               const float* g_opacity, float* g_log_scales, float* g_logit_opacity, int accumulate,
                               void* stream) {
  if (n < 0 || (n > 0 && (!scales || !opacity || !g_scales || !g_opacity || !g_log_scales || !g_logit_opacity)))
    return fail(TS_ERR_ARG, "ts_activate_backward: bad argument");
  launch_activate_bwd(scales, opacity, g_scales, g_opacity, n, g_log_scales, g_logit_opacity, accumulate,
                      (cudaStream_t)stream);
  TS_CHECK_LAUNCH();
  return TS_OK;
}

ts_status ts_l1_loss(const float* rgba, const float* target, int64_t n_pixels, float* loss_out, float* dL_drgba,
                     void* stream) {
  if (!rgba || !target || !loss_out || !dL_drgba || n_pixels < 0) return fail(TS_ERR_ARG, "ts_l1_loss: bad argument");
  ProfScope p((cudaStream_t)stream, "l1_loss");
  launch_l1_loss(reinterpret_cast<const float4*>(rgba), reinterpret_cast<const float4*>(target), n_pixels, loss_out,
                 reinterpret_cast<float4*>(dL_drgba), (cudaStream_t)stream);
  TS_CHECK_LAUNCH();
  return TS_OK;
}

}  // extern "C"
