/*
 * texsplat.h -- C ABI of the B300 textured 2D-Gaussian-splat renderer.
 *
 * The library renders planar (2DGS) Gaussian splats that each carry a T x T
 * texture of 8 material channels, composites the texture lookups into a
 * G-buffer and shades it against a cube-map environment (TextureSplat,
 * Sec. 3), and differentiates all of it.  Every entry point takes plain
 * pointers and sizes; no C++ or framework type crosses this boundary.
 *
 * Conventions shared by all entry points
 *   - Every call returns a ts_status; TS_OK is 0.  On failure the call has
 *     no partial effect on caller buffers unless stated, and
 *     ts_last_error() returns a message (thread-local, valid until the next
 *     call on that thread).  No exception or abort crosses the ABI.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued in stream order.  Device pointers must
 *     belong to the scene's device.
 *   - Arrays are dense, row-major, float32 unless stated.
 *   - Channel order of a texel (8 channels): 0..2 albedo RGB, 3 metallic,
 *     4 roughness, 5..7 tangent-space normal (x, y, z) (Sec. 3.5.1).
 *   - Texture layout [n][T][T][8]: row index along the splat's v axis
 *     (texture t), column along u (texture s) (Eq. 5).
 *   - Cube maps [6][R][R][3]: faces +x,-x,+y,-y,+z,-z, row t, column s, in
 *     the OpenGL/CUDA cube-face convention.
 */
#ifndef TEXSPLAT_H
#define TEXSPLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int ts_status;
#define TS_OK 0
#define TS_ERR_ARG 1      /* invalid argument (null pointer, bad size, bad enum) */
#define TS_ERR_OOM 2      /* device or host allocation failed */
#define TS_ERR_CAPACITY 3 /* a fixed-capacity buffer would overflow */
#define TS_ERR_CUDA 4     /* a CUDA runtime call failed (message has the CUDA error) */
#define TS_ERR_TIMEOUT 5  /* a wait ran out of time (host side, or a bounded wait inside a sort) */
#define TS_ERR_STATE 6    /* call out of order (e.g. render before upload) */

typedef enum ts_dtype { TS_F32 = 0, TS_BF16 = 1, TS_F16 = 2 } ts_dtype;

/* Pinhole camera, OpenCV axes (x right, y down, z forward).  R is the
 * world->camera rotation (row-major), t the world->camera translation, so a
 * world point X maps to R X + t.  Pixel centres are at (i + 0.5, j + 0.5).
 * width, height >= 1.  visibility: NULL, or a caller-owned device array
 * [height][width] of the view's visibility V in [0, 1] (Eq. 12: the specular
 * light is V C_spec + (1 - V) L_ind); read by the render and, for a saved
 * render, by its backward, so it must stay valid until both ran.  V and
 * L_ind form the indirect-light model together: it applies to scenes with
 * per-splat SH (ts_upload_indirect); for a scene without SH the plain model
 * renders (V = 1, L_ind = 0) and visibility is not read. */
typedef struct ts_camera {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  int32_t width, height;
  const float* visibility;
} ts_camera;

typedef struct ts_scene ts_scene;  /* library-owned splats, texels, environment */
typedef struct ts_saved ts_saved;  /* library-owned forward state for the backward */

/* Caller-owned device buffers receiving gradients.  The backward ACCUMULATES
 * (+=) into every non-NULL pointer; NULL skips that group.  Shapes follow
 * the uploads: means [n][3], quats [n][4] (w,x,y,z; gradient w.r.t. the
 * uploaded, unnormalised quaternion), scales [n][2] (linear), opacity [n]
 * (linear), texels [n][T][T][8] (float32 whatever the stored dtype), spec
 * (all mip levels concatenated, [6][R_l][R_l][3] each), irr [6][R][R][3],
 * sh [n][K][3] (the indirect-light SH coefficients, K = (degree + 1)^2). */
typedef struct ts_grads {
  float* means;
  float* quats;
  float* scales;
  float* opacity;
  float* texels;
  float* spec;
  float* irr;
  float* sh;
} ts_grads;

/* Fragment statistics of one forward (for roofline accounting). */
typedef struct ts_frag_stats {
  int64_t n_pairs;      /* (tile, splat) pairs after binning */
  int64_t n_evaluated;  /* (pixel, splat) fragments tested before each pixel terminated */
  int64_t n_blended;    /* fragments that passed the support and alpha tests and were blended */
  int64_t n_visible;    /* splats that survived culling */
  int64_t n_texels_read;   /* distinct (list item, texel) pairs read by blended fragments: each blended
                              fragment reads its four bilinear corners (Eq. 6), clamped to the chart */
  int64_t n_items_blended; /* distinct list items (splats of a view) blended at some pixel */
} ts_frag_stats;

/* ---- scenes --------------------------------------------------------------- */

/* Creates an empty scene on CUDA device `device`. *out owns device memory
 * until ts_destroy_scene. */
ts_status ts_create_scene(ts_scene** out, int device);
ts_status ts_destroy_scene(ts_scene* scene);

/* Splat geometry of Sec. 3.1 (Eq. 1): means p [n][3], quaternions [n][4]
 * (w,x,y,z, normalised inside), linear scales (s_u, s_v) [n][2] > 0 and
 * linear opacities o [n] in [0,1].  Copies into library memory (from device
 * memory if src_on_device, else host memory; the call then returns after
 * the host buffers may be reused).  n >= 0 (0 renders an empty image).
 * Replaces previous geometry; the atlas must be re-uploaded if n changed.
 * The values are checked on the device before they replace anything:
 * TS_ERR_ARG (message: the count, the first bad index and the reasons) for
 * a non-finite centre, a quaternion that is non-finite or of squared norm
 * below 1e-20, a scale that is non-finite or <= 0, an opacity outside
 * [0, 1] or NaN.  On every error (TS_ERR_ARG, TS_ERR_OOM, TS_ERR_CUDA) the
 * scene keeps its previous geometry and no library memory is left behind.
 * Synchronises `stream`. */
ts_status ts_upload_gaussians(ts_scene* scene, int64_t n, const float* means, const float* quats,
                              const float* scales, const float* opacity, int src_on_device,
                              void* stream);

/* Per-primitive textures (Sec. 3.2-3.3; packed as in the supplementary's
 * atlas construction, one contiguous T x T chart per splat).  texels
 * [n][T][T][C] float32 with C == 8 and 1 <= T <= 32; `store` selects the
 * stored precision (float32, or bfloat16 / float16 rounded to nearest
 * even).  Lookups always widen to float32.  Texel values are data and are
 * not checked.  On error the previous atlas stays in place.  Synchronises
 * `stream`. */
ts_status ts_upload_atlas(ts_scene* scene, int T, int C, ts_dtype store, const float* texels,
                          int src_on_device, void* stream);

/* Environment light of Sec. 3.5.4 (Eq. 11-12): `levels` specular mips, level l
 * of resolution max(1, base_res >> l), concatenated [6][R_l][R_l][3]; the
 * irradiance cube [6][irr_res][irr_res][3]; the split-sum BRDF table
 * [lut_res][lut_res][2] (row = roughness, column = N.w_o; channels scale,
 * bias).  `store` F32 or F16 for the cube maps (the table stays float32).
 * 1 <= levels <= 12.  On error the previous environment stays in place.
 * Synchronises `stream`. */
ts_status ts_upload_envmap(ts_scene* scene, int levels, int base_res, const float* spec, int irr_res,
                           const float* irr, int lut_res, const float* lut, ts_dtype store,
                           int src_on_device, void* stream);

/* ---- rendering -------------------------------------------------------------- */

/* Renders one view: cull and bin the splats into 16x16 tiles, sort each
 * tile's list by depth (keys bit-exact with the FP32 binning specification),
 * intersect each pixel ray with each listed splat in closed form to get its
 * local (u, v) (Sec. 3.1, Eq. 2), fetch the bilinear texel (Eq. 5-6),
 * rotate the tangent normal to world space (Eq. 7), composite front to back
 * into the G-buffer (Eq. 3, Eq. 8-9) and shade it (Eq. 10-12).
 * out_rgba: caller-owned device buffer [H][W][4] (RGB colour, alpha = 1 - T).
 * saved: NULL for inference; otherwise receives a handle holding what the
 * backward needs (release with ts_release_saved).  Synchronises the stream
 * once to size the pair buffer (see ts_render_views for the batched form). */
ts_status ts_render(ts_scene* scene, const ts_camera* cam, float* out_rgba, ts_saved** saved,
                    void* stream);

/* Batched form: n_views views, view i of scenes[i] with cams[i] into
 * out_rgba[i].  All views share one binning/sort/raster launch sequence.
 * saved may be NULL.  1 <= n_views <= 32.  Errors: TS_ERR_ARG (bad
 * arguments, mixed dtypes / samplers / normal encodings in one batch),
 * TS_ERR_STATE (missing or stale uploads, a sampler that cannot save state),
 * TS_ERR_CAPACITY (more than 2^30 (tile, splat) pairs or a batch too large),
 * TS_ERR_TIMEOUT (the bounded inter-block wait of the per-splat depth sort
 * ran out -- a device-side failure, reported at this call's
 * synchronisation, before any pair is emitted), TS_ERR_OOM, TS_ERR_CUDA.
 * The pair sort waits on nothing.  The rasterisers take the tiles longest
 * list first; if the bounded wait of that launch-order sort runs out, they
 * take the tiles in tile order instead, which changes no result, so an image
 * returned with TS_OK is always the one the lists define.  (Should a kernel
 * after the synchronisation still find a list id out of range, the image is
 * written as NaN and the next call reports TS_ERR_TIMEOUT.) */
ts_status ts_render_views(ts_scene* const* scenes, const ts_camera* cams, int n_views,
                          float* const* out_rgba, ts_saved** saved, void* stream);

/* Backward of ts_render / ts_render_views through shading, compositing,
 * texel fetch and intersection (Sec. 3.6 optimises all of these).
 * dL_drgba: device [H][W][4] per view (array of n_views pointers for the
 * batched form, in view order).  Gradients are accumulated into `grads`
 * (one set per scene; for the batched form all views must share one scene).
 * The saved handle stays valid (backward may be repeated).  The backward
 * recomputes each fragment from the scene's current splats, texels and
 * environment (only the lists and per-pixel state are saved), so the scene
 * must not change between the forward and its backward: update parameters
 * after the backward (as api.Trainer and the autograd wrapper do).  An upload
 * that replaced a scene's buffers since the forward (ts_upload_gaussians,
 * ts_upload_atlas, ts_upload_envmap, a new SH degree or count) makes this
 * call return TS_ERR_STATE instead of reading the freed buffers; a scene must
 * outlive its saved states.  The
 * backward rasteriser takes the tiles by the list entries it walks (up to
 * each pixel's last blended entry), longest first; temporaries are allocated
 * with cudaMallocAsync on `stream`. */
ts_status ts_render_backward(const ts_saved* saved, const float* const* dL_drgba,
                             const ts_grads* grads, void* stream);

ts_status ts_release_saved(ts_saved* saved);

/* ---- inspection of a saved forward (tests and accounting) ------------------ */

/* Number of pairs and tiles (global, over all views) of a saved forward.
 * Synchronises the saved forward's stream. */
ts_status ts_saved_sizes(const ts_saved* saved, int64_t* n_pairs, int64_t* n_tiles);

/* Copies the sorted per-tile lists to caller device buffers:
 * item_ids [n_pairs] (splat id + the view's item offset), tile_ranges
 * [n_tiles][2] (start, end), depth_bits [n_items] (float bits of each
 * splat's camera depth, 0xFFFFFFFF when culled).  Any pointer may be NULL. */
ts_status ts_saved_copy_lists(const ts_saved* saved, uint32_t* item_ids, uint32_t* tile_ranges,
                              uint32_t* depth_bits, void* stream);

/* Copies view v's per-pixel forward state: gbuf [H][W][8] (blended X of
 * Eq. 9), trans [H][W] (final transmittance T), last [H][W] (index in the
 * pair list of the last blended fragment, -1 if none).  NULL skips. */
ts_status ts_saved_copy_pixels(const ts_saved* saved, int view, float* gbuf, float* trans,
                               int32_t* last, void* stream);

/* Fragment counts of a saved forward (counted by a separate, untimed pass
 * over the same lists; the texel counts use a temporary bitmap of one bit
 * per texel of every list item's chart).  Synchronises the stream. */
ts_status ts_saved_frag_stats(const ts_saved* saved, ts_frag_stats* out, void* stream);

/* Geometry size, texture resolution and stored atlas dtype of a scene (any
 * pointer may be NULL).  TS_ERR_STATE if geometry or atlas is missing. */
ts_status ts_scene_info(const ts_scene* scene, int64_t* n, int* T, int* dtype);

/* ---- training: optimiser step and in-place scene updates ------------------------ */

/* Adam (Kingma & Ba) hyper-parameters; step >= 1 is the 1-based update count
 * used for the bias corrections. */
typedef struct ts_adam {
  float lr, beta1, beta2, eps;
  int64_t step;
} ts_adam;

/* One Adam step on n float32 master parameters `param` with gradient `grad`
 * and moments m, v (all device, 16-byte aligned, updated in place).  If
 * zero_grad, `grad` is zeroed after use (the backward accumulates).  If
 * `shadow` is non-NULL the updated parameters are also written there in
 * `shadow_dtype` (float32, or bfloat16 / float16 rounded to nearest even) --
 * e.g. the scene's stored atlas from ts_scene_texels, so training keeps
 * float32 masters while rendering reads the reduced-precision copy.
 * Stream-ordered, no synchronisation. */
ts_status ts_adam_update(float* param, float* grad, float* m, float* v, int64_t n, const ts_adam* hp, void* shadow,
                         ts_dtype shadow_dtype, int zero_grad, void* stream);

/* Device pointer, resolution and dtype of a scene's stored atlas
 * ([n][T][T][8] in that dtype); valid until the atlas is re-uploaded. */
ts_status ts_scene_texels(ts_scene* scene, void** texels, int* T, int* dtype);

/* Device pointers and dtype (TS_F32 or TS_F16) of a scene's stored
 * environment: the specular cube levels back to back in the layout of
 * ts_upload_envmap (level l at offset sum_{k<l} 6 r_k^2 3 elements) and the
 * irradiance cube -- the same element order as the gradients of ts_grads
 * (spec, irr), so ts_adam_update can write its shadow copy there.  Valid
 * until the environment is re-uploaded.  TS_ERR_STATE if none is. */
ts_status ts_scene_envmap(ts_scene* scene, void** spec, void** irr, int* dtype);

/* Image term of the training loss (Sec. 3.6) over the RGB channels of
 * [height][width][4] float32 device images (alpha ignored):
 *   *loss = (1 - lambda) L1 + lambda (1 - SSIM),
 * L1 = mean |rgba - target|, SSIM = mean structural similarity under an
 * 11x11 Gaussian window (sigma 1.5, zero padding, C1 = 0.01^2,
 * C2 = 0.03^2); the paper uses lambda = 0.2.  Writes the scalar to the
 * device float `loss` and dL/drgba (alpha column 0) to `grad` (overwritten,
 * not accumulated).  Stream-ordered; allocates its 36 B/pixel scratch with
 * cudaMallocAsync on `stream`.  Errors: TS_ERR_ARG (NULL pointers, empty or
 * > 2^28-pixel image, lambda outside [0, 1]), TS_ERR_CUDA. */
ts_status ts_image_loss(const float* rgba, const float* target, int width, int height, float lambda_dssim,
                        float* loss, float* grad, void* stream);

/* Copies view v's blended camera depth zsum [H][W] (sum over blended
 * fragments of alpha T z, z the camera depth of the ray-splat hit) and
 * coverage acc [H][W] (sum of alpha T) of a saved render.  The expected
 * depth is zsum / acc.  NULL skips. */
ts_status ts_saved_copy_depth(const ts_saved* saved, int view, float* zsum, float* acc, void* stream);

/* Normal-consistency loss of Sec. 3.6 on view `view` of a saved render:
 *   *loss = weight * L_n,  L_n = sum over counted pixels of (1 - N~ . N^)
 *                               / ((W - 2)(H - 2)),
 * N^ the normalised blended normal channel, N~ the normal of the depth map:
 * the expected depth zsum / acc back-projected through the camera, central
 * differences of the 4 neighbours, cross product facing the camera, in
 * world space.  A pixel counts when it is interior, it and its neighbours
 * have coverage >= 0.5 and its normal and cross product are non-zero.
 * Stores the loss's gradient w.r.t. the view's normal channels, coverage
 * and blended depth in the saved state (overwriting an earlier call); the
 * next ts_render_backward of `saved` adds them to the image gradient, so
 * the backward differentiates L_img + weight L_n.  Writes the device float
 * `loss`; stream-ordered (first call on a view allocates its buffers).
 * Errors: TS_ERR_ARG (NULL, bad view, negative weight), TS_ERR_CUDA. */
ts_status ts_normal_loss(ts_saved* saved, int view, float weight, float* loss, void* stream);

/* ---- indirect light (Eq. 9, Eq. 12) ---------------------------------------- */

/* Per-splat indirect light: real SH coefficients of degree 0, 1 or 2 (the
 * convention of 3DGS: K = 1, 4 or 9 basis functions), [n][K][3] float32 (RGB
 * per basis function), copied to library memory (src_on_device selects the
 * source side).  Each blended fragment evaluates its splat's SH in the
 * reflection direction of its own normalised normal and the results are
 * blended as a G-buffer channel L_ind; the pixel's visibility (ts_camera)
 * mixes it into the specular light.  degree = -1 (coeffs ignored) removes
 * the SH.  Renders of a scene with SH need the software sampler.  A first
 * upload (or one that changes the degree or the splat count) allocates and
 * synchronises `stream`; a re-upload of the same degree and count from
 * device memory overwrites the coefficients in place, stream-ordered
 * without synchronisation (training updates).  Errors: TS_ERR_ARG (NULL scene, degree
 * outside [-1, 2], NULL coeffs), TS_ERR_STATE (no geometry), TS_ERR_OOM,
 * TS_ERR_CUDA. */
ts_status ts_upload_indirect(ts_scene* scene, int degree, const float* coeffs, int src_on_device, void* stream);

/* ---- hardware-texture atlas (test-time sampling) ------------------------- */

/* Texture samplers of the forward render (ts_scene_set_sampler). */
enum { TS_SAMPLER_SOFTWARE = 0, TS_SAMPLER_HW_ATLAS = 1, TS_SAMPLER_FLAT = 2 };

/* Chart orders of ts_scene_build_atlas2d. */
enum { TS_PACK_SPLAT_ID = 0, TS_PACK_MORTON = 1 };

/* Builds the 2-D texture atlases of supplementary Sec. 1 ("Texture Atlas"):
 * the scene's T x T charts packed row-major into two 4-channel
 * 2-D textures (channels 0-3: albedo, metallic; 4-7: roughness, tangent
 * normal), each a CUDA array sampled through a texture object with linear
 * filtering and clamp addressing, plus the indirection buffer splat -> chart
 * origin.  The atlas is near square with a power-of-two width (so texel
 * coordinates stay small and exact in FP32).  store: TS_F32 (16 B per texel
 * per atlas) or TS_F16 (8 B).  packing: TS_PACK_SPLAT_ID places charts in
 * splat id order (the paper's unordered packing); TS_PACK_MORTON in the
 * Morton order of the splat centres (30-bit code in the centres' bounding
 * box), so splats near each other in space get neighbouring charts -- the
 * locality-aware packing the paper names as future work.  Reads the stored
 * texels as they are now: an
 * atlas upload invalidates it (TS_ERR_STATE on a hardware-sampled render
 * until rebuilt); in-place texel updates through ts_scene_texels do not, so
 * rebuild after them.  Synchronises `stream`.  Errors: TS_ERR_ARG (NULL
 * scene, other store), TS_ERR_STATE (no or stale texels), TS_ERR_CAPACITY
 * (more charts than the device's largest 2-D surface holds), TS_ERR_OOM,
 * unknown packing TS_ERR_ARG,
 * TS_ERR_CUDA.  Library-owned; freed with the scene. */
ts_status ts_scene_build_atlas2d(ts_scene* scene, ts_dtype store, int packing, void* stream);

/* Selects how forward renders of `scene` sample its textures:
 *   TS_SAMPLER_SOFTWARE (default): bilinear filter (Eq. 6) in FP32 from the
 *     per-splat chart layout -- the parity path, with backward;
 *   TS_SAMPLER_HW_ATLAS: tex2D on the 2-D atlases (needs
 *     ts_scene_build_atlas2d); the texture unit's bilinear weights have 8
 *     fractional bits, so results differ from the definition by up to about
 *     2^-9 of the texel differences per axis (a reported-error path);
 *   TS_SAMPLER_FLAT: one attribute vector per splat (texel (0, 0) of its
 *     chart) without texture lookup: the untextured baseline the paper's
 *     Table 3 compares against.
 * The hardware and flat samplers are inference-only: a render that asks for
 * saved state returns TS_ERR_STATE, as does a batch whose scenes use
 * different samplers (TS_ERR_ARG).  Returns TS_ERR_ARG for an unknown value. */
ts_status ts_scene_set_sampler(ts_scene* scene, int sampler);

/* Tangent-normal encodings of the texture channels 5-7 (Sec. 3.5.1). */
enum { TS_NORMAL_XYZ = 0, TS_NORMAL_XY = 1 };

/* Selects how the scene's textures hold the tangent normal n^t:
 *   TS_NORMAL_XYZ (default): channels 5-7 store the three signed components;
 *   TS_NORMAL_XY: channels 5-6 store (n_x, n_y) and the renderer rebuilds
 *     n_z = sqrt(max(0, 1 - n_x^2 - n_y^2)) from the bilinearly interpolated
 *     pair (Sec. 3.5.1); channel 7 is never read and its gradient is zero.
 * The texel keeps its 8-channel stride either way (16-byte aligned vector
 * loads), so the encoding changes what is rendered, not the atlas size.
 * Applies to every sampler and to the backward.  All scenes of one batch
 * must share the encoding (TS_ERR_ARG).  Returns TS_ERR_ARG for NULL or an
 * unknown value. */
ts_status ts_scene_set_normal_encoding(ts_scene* scene, int encoding);

/* Overwrites the scene's geometry (same n as uploaded) from device arrays,
 * stream-ordered without synchronisation (for updates between training
 * steps).  Layouts as in ts_upload_gaussians. */
ts_status ts_scene_set_geometry(ts_scene* scene, const float* means, const float* quats, const float* scales,
                                const float* opacity, void* stream);

/* ---- serving: continuous batching of view requests ------------------------------ */

typedef struct ts_server ts_server;

typedef struct ts_serve_stats {
  int64_t submitted, completed, rejected, failed, batches;
  double mean_batch;      /* views per launched batch */
  double p50_ms, p99_ms;  /* latency, submission -> completion of the batch's last kernel */
  double mean_ms;
  double fps;             /* completed views / (last completion - first submission) */
  double mpix_per_s;
  int64_t true_ups;       /* batches whose counted pairs needed more memory than their estimate */
  int64_t over_budget;    /* of those, batches that went past the budget because waiting could not end */
  double peak_reserved_bytes;  /* largest memory reservation held at once (outputs + render buffers) */
} ts_serve_stats;

/* Starts a view server on `device` with n_streams worker threads (one CUDA
 * stream each, 1..16), batches of at most max_batch views (1..32), and a
 * device-memory budget of arena_bytes (> 0) for requests in flight.  A
 * request is admitted with its output, the render's exact per-splat
 * buffers and an estimate of its (tile, splat) pair buffers -- pairs per
 * pixel learned per scene as the largest value its renders showed, 32
 * before the first.  When the batch has counted its pairs (the render's one
 * synchronisation) its reservation is trued up to the exact bytes it still
 * allocates: a surplus is returned at once, a deficit waits for running
 * batches to free memory (if every running batch is waiting, it proceeds and
 * is counted in over_budget, since memory held by uncollected results can
 * only come back through ts_server_wait); a batch that alone exceeds the
 * budget fails with TS_ERR_CAPACITY, and so does a queued request that its
 * scene's learned pair count puts above the whole budget (reported by
 * ts_server_wait, counted as failed).  Scenes stay resident: requests name a
 * scene created and uploaded beforehand; it must outlive its requests. */
ts_status ts_server_create(ts_server** out, int device, size_t arena_bytes, int n_streams, int max_batch);

/* Stops the workers (queued requests are dropped) and frees everything. */
ts_status ts_server_destroy(ts_server* server);

/* Queues one view (forward render, no backward state) and returns a ticket
 * at once.  A worker that becomes free takes every queued request that fits
 * -- same atlas dtype, within max_batch and the memory budget -- into one
 * batched launch sequence (ts_render_views); requests arriving meanwhile
 * join the next batch.  TS_ERR_CAPACITY if the request alone exceeds the
 * budget (counted as rejected). */
ts_status ts_server_submit(ts_server* server, ts_scene* scene, const ts_camera* cam, uint64_t* ticket);

/* Waits up to timeout_s seconds for a ticket (TS_ERR_TIMEOUT, ticket kept),
 * then copies its RGBA image [H][W][4] to out_rgba (device memory if
 * out_on_device, else host; NULL discards) and retires the ticket.  The
 * image is identical to ts_render's for the same scene and camera. */
ts_status ts_server_wait(ts_server* server, uint64_t ticket, float* out_rgba, int out_on_device,
                         double timeout_s);

/* Latency / throughput counters since creation or the last reset. */
ts_status ts_server_stats(ts_server* server, ts_serve_stats* out);

/* The bytes a request for `scene` and `cam` would be admitted with now
 * (output, the render's per-splat buffers, the current pair estimate). */
ts_status ts_server_request_bytes(ts_server* server, ts_scene* scene, const ts_camera* cam, size_t* bytes);

/* The device-time interval of each of the last batches (at most
 * max_entries, oldest first, up to 4096 kept since the last reset): the
 * worker that ran it, its view count and its start / end in ms on the GPU
 * clock, measured by CUDA events on the worker's stream against an event
 * recorded when the server was created.  Intervals of different workers
 * that intersect ran on the device at the same time.  *n_out receives the
 * count.  TS_ERR_ARG for NULL outputs. */
ts_status ts_server_batch_log(ts_server* server, int32_t max_entries, int32_t* n_out, int32_t* worker,
                              int32_t* views, double* t0_ms, double* t1_ms);
ts_status ts_server_reset_stats(ts_server* server);

/* ---- training helpers --------------------------------------------------------- */

/* L1 image loss over the RGB channels: loss_out[0] = mean |rgba - target|
 * (device scalar, written, not accumulated), dL_drgba = sign(rgba - target) /
 * (3 H W) for RGB and 0 for alpha (written).  n_pixels = H * W. */
ts_status ts_l1_loss(const float* rgba, const float* target, int64_t n_pixels, float* loss_out,
                     float* dL_drgba, void* stream);

/* Activations of the raw optimisation variables, so that the render ABI
 * sees linear values: scales[i] = exp(log_scales[i]) for the n x 2 scale
 * components, opacity[k] = 1 / (1 + exp(-logit_opacity[k])) for the n
 * opacities (the parameterisation the optimisation of Sec. 3.6 runs on;
 * quaternions need none: the renderer normalises them and its gradient is
 * w.r.t. the raw quaternion).  Device arrays, stream-ordered.
 * TS_ERR_ARG for n < 0 or a NULL array with n > 0. */
ts_status ts_activate(int64_t n, const float* log_scales, const float* logit_opacity, float* scales, float* opacity,
                      void* stream);

/* Chain rule of ts_activate: g_log_scales = g_scales * scales,
 * g_logit_opacity = g_opacity * opacity * (1 - opacity), from the activated
 * values; written, or added when accumulate != 0. */
ts_status ts_activate_backward(int64_t n, const float* scales, const float* opacity, const float* g_scales,
                               const float* g_opacity, float* g_log_scales, float* g_logit_opacity, int accumulate,
                               void* stream);

/* Self-test of the failure path of the radix sort's inter-block wait: runs
 * one sort pass whose only block waits on a block that never runs, so its
 * bounded wait (about a second) runs out; the pass sets the device flag the
 * renders read, and this call reads and clears it.  Returns TS_ERR_TIMEOUT
 * when the wait ran out and was reported (the expected result; the device
 * stays usable), TS_ERR_STATE if it was not reported, TS_ERR_CUDA on a CUDA
 * error.  Synchronises `stream`. */
ts_status ts_selftest_sort_wait(int device, void* stream);

/* Host-side failure injection for tests: with after = k >= 0, the (k+1)-th
 * device allocation the library makes from now on (uploads, render and
 * backward scratch) fails once as out of memory, so that error paths can be
 * exercised without exhausting the device; after = -1 disarms it.  No GPU
 * fault is involved.  TS_ERR_ARG for after < -1. */
ts_status ts_debug_fail_alloc(int64_t after);

/* ---- rendering without device allocation ------------------------------------ */

/* The paper has no counterpart of this entry point; it serves callers that
 * cannot allocate device memory while they render: a renderer embedded in a
 * host application that owns the whole device budget, a real-time frame
 * loop that cannot accept an allocation's latency or failure, or a plugin
 * that may only touch the buffers it is handed.
 *
 * Same forward render as ts_render (identical kernels and results), but
 * every input is a caller device buffer and the call allocates nothing: no
 * cudaMalloc / cudaFree / allocating library call.  Its working set lives in
 * one fixed device array of about 21 MB compiled into the library, which
 * every GPU that loads the library holds until the process exits.
 *   Limits: n <= 32768 splats, at most 8192 16x16 tiles (1920x1080 fits),
 *   at most 1048576 (tile, splat) pairs after binning; beyond them the call
 *   returns TS_ERR_CAPACITY (the pair limit is found after binning, so the
 *   output is then left unwritten).
 *   Inputs: means [n][3], quats [n][4] (16-byte aligned), scales [n][2]
 *   (8-byte aligned), opacity [n], texels [n][T][T][8] float32 (16-byte
 *   aligned), the environment as in ts_upload_envmap in float32 (spec
 *   levels concatenated), camera by value, out_rgba [H][W][4].
 *   It renders the default model: three stored tangent-normal components,
 *   no indirect light (the camera's visibility is ignored), the software
 *   sampler.
 *   The first call on a device looks up the array's device address (once
 *   per device, with that device current): make that first call before any
 *   stream capture.  Every call shares the array: the call clears what must
 *   start at zero, and calls that overlap on the GPU (streams not ordered
 *   with each other) race on it.  The call synchronises `stream` once to
 *   read the pair count and the sort flags: TS_ERR_TIMEOUT when the depth
 *   sort's bounded wait ran out (the output is then left unwritten); the
 *   launch-order sort falls back to tile order as in ts_render_views. */
ts_status ts_render_noalloc(int64_t n, const float* means, const float* quats, const float* scales,
                            const float* opacity, int T, const float* texels, int levels, int base_res,
                            const float* spec, int irr_res, const float* irr, int lut_res, const float* lut,
                            const ts_camera* cam, float* out_rgba, void* stream);

/* ---- accounting and stage timing ------------------------------------------- */

/* Number of kernels this library has launched since it was loaded (all
 * threads, all devices). */
int64_t ts_launch_count(void);

/* Turns per-stage CUDA-event timing on (1) or off (0).  While on, each
 * pipeline stage (preprocess, sort_splats, scan_counts, emit_pairs,
 * sort_pairs, tile_ranges, raster_fwd, shade_bwd, raster_bwd,
 * preprocess_bwd, l1_loss, adam) records an event pair on the stream it
 * runs on. */
ts_status ts_profile_enable(int on);

/* Waits for the recorded events, writes one line per stage
 * "name launches total_ms\n" into buf (NUL-terminated, truncated to buflen)
 * and clears the records. */
ts_status ts_profile_report(char* buf, size_t buflen);

/* Measures the device's FP32 FMA rate in TFLOP/s (2 FLOP per FMA), the
 * denominator of the rasterisers' arithmetic roofline: independent fmaf
 * chains (*scalar_tflops) and float2 fma pairs (*paired_tflops) on every
 * lane of a full-occupancy grid, best of three ~10 ms runs after a warm-up.
 * Runs on the legacy default stream of `device` and synchronises it;
 * allocates and frees a small device buffer.  Not part of the paper's
 * method: a measurement utility.  Returns TS_ERR_ARG for null outputs,
 * TS_ERR_CUDA on any CUDA error. */
ts_status ts_measure_fp32_peak(int device, double* scalar_tflops, double* paired_tflops);

/* ---- errors ---------------------------------------------------------------- */

const char* ts_last_error(void);
const char* ts_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TEXSPLAT_H */
