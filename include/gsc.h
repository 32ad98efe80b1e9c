/*
 * gsc.h - C ABI of the B300 structured-3DGS frame renderer (GS-Cache path).
 *
 * One context renders frames of structured 3D Gaussian Splatting models
 * (anchors with a feature vector, decoded by small MLPs into k "neural
 * Gaussians" each) on one GPU.  A frame runs, entirely in the library's own
 * CUDA kernels:
 *   1. anchor filtering: frustum + distance LOD            (Sec. 3.2, Alg. 1)
 *   2. derivation: MLP(feature, view direction) -> Gaussians (Eq. 3, Sec. 6),
 *      optionally reusing cached results across frames   (Sec. 4, Alg. 1, Eq. 4)
 *      and sharing one derivation between two eyes        (Eq. 5-6)
 *   3. splatting: EWA projection, exact tile coverage, key generation,
 *      radix sort, front-to-back alpha blending            (Eq. 1-2, Sec. 3.1, Sec. 6)
 *
 * Conventions
 *  - Every call returns a gsc_status (0 = GSC_OK).  Nothing throws across the
 *    ABI.  On error gsc_last_error() returns a message for the context.
 *  - The context owns every internal device buffer.  Output images are
 *    caller-owned device memory (gsc_render_frame) or host memory
 *    (gsc_render_frame_host).
 *  - All work is enqueued on the CUDA stream given to gsc_create (NULL = the
 *    legacy default stream).  gsc_render_frame with stats == NULL is
 *    asynchronous; see its comment for deferred errors.
 *  - Sizes fixed by this build: feature dim 32, k = 10 Gaussians per anchor,
 *    MLP hidden width 32, three heads (opacity k, colour 3k, covariance 7k).
 *  - A context is not thread-safe; use one per host thread.
 */
#ifndef GSC_H
#define GSC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GSC_API __attribute__((visibility("default")))
#else
#define GSC_API
#endif

#define GSC_VERSION 1
#define GSC_FEAT_DIM 32
#define GSC_K 10
#define GSC_HIDDEN 32
#define GSC_MAX_VIEWS 32

typedef struct gsc_ctx gsc_ctx;

typedef enum {
  GSC_OK = 0,
  GSC_ERR_INVALID_ARG = -1,   /* null pointer, bad size, unsupported dims */
  GSC_ERR_OOM = -2,           /* device or pinned-host allocation failed */
  GSC_ERR_CUDA = -3,          /* a CUDA runtime call failed (message has the name) */
  GSC_ERR_CAPACITY = -4,      /* pair buffer overflowed in an asynchronous frame; grown, re-render */
  GSC_ERR_TIMEOUT = -5,       /* a bounded device-side wait gave up; frame output invalid */
  GSC_ERR_STATE = -6,         /* call out of order (e.g. render before set_cameras) */
  GSC_ERR_UNIMPLEMENTED = -7, /* requested form not built */
  GSC_ERR_INTERNAL = -8
} gsc_status;

typedef enum { GSC_PREC_FP32 = 0, GSC_PREC_BF16 = 1, GSC_PREC_FP8 = 2 } gsc_precision;

/* Image format of the outputs.  F32: float [H][W][3], the blended colour
 * C + T bg.  RGBA8: uint8 [H][W][4], round-to-nearest-even of 255 x the same
 * colour clamped to [0, 1], and alpha = that of 1 - T (the display format:
 * 4 bytes per pixel instead of 12). */
typedef enum { GSC_OUT_F32 = 0, GSC_OUT_RGBA8 = 1 } gsc_out_format;

/* Guiding function H of Eq. 4: the reuse depth of the next frame from this
 * frame's update rate u = misses / visible anchors of a derivation view
 * (depth reuse form; D = max_depth; the result is clamped to [1, D]).
 * LINEAR (the paper's experiments): round(D (1 - u)), in integers, halves up.
 * EXP (for accelerating motion): round(D^(1 - u)), in float64; it falls
 *   faster than the linear one as u grows and meets it at u = 0 and u = 1.
 * STAGED (for staged speed changes): D for u < 0.1, ceil(D / 2) for
 *   u < 0.3, 1 otherwise, in integers.
 * The paper names the exponential and staged responses without a formula;
 * these are this library's forms of them. */
typedef enum { GSC_GUIDE_LINEAR = 0, GSC_GUIDE_EXP = 1, GSC_GUIDE_STAGED = 2 } gsc_depth_guide;

typedef enum {
  GSC_REUSE_OFF = 0,      /* decode every visible anchor every frame */
  GSC_REUSE_DEPTH = 1,    /* Alg. 1 dynamic cache depth (Eq. 4, linear guide) */
  GSC_REUSE_LEARNED = 2   /* learned per-anchor reuse predictor (gsc_reuse_*); lines past D_max stay invalid */
} gsc_reuse_mode;

/* flags */
#define GSC_FLAG_DEBUG_ATTRS 0x1u  /* keep derived attributes for gsc_debug_attrs */
#define GSC_FLAG_DEBUG_T 0x2u      /* keep per-pixel final transmittance */
#define GSC_FLAG_TIMING 0x4u       /* per-stage CUDA-event timing into gsc_frame_stats */
#define GSC_FLAG_REUSE_COLLECT 0x8u /* reuse forms: record predictor inputs + labels (gsc_reuse_collect) */
#define GSC_FLAG_BLEND_WORK 0x10u  /* blend counts its work per frame (gsc_debug_blend_work); slower */
#define GSC_FLAG_UNFUSED 0x20u     /* FP32 only: the derivation as separate operators through device memory
                                      (gather, GEMM, ReLU, GEMM, split, activation): the ablation's decoder
                                      without fused kernels; the same arithmetic as the fused one */

enum { GSC_STEREO_OFF = 0, GSC_STEREO_UNIFIED = 1, GSC_STEREO_EXACT = 2 };

typedef struct {
  uint32_t max_views;        /* cameras per frame, 1..GSC_MAX_VIEWS */
  uint32_t precision;        /* gsc_precision of the derivation MLPs */
  uint32_t reuse;            /* gsc_reuse_mode */
  uint32_t stereo_unify;     /* cameras with a stereo partner share one derivation from the Eq. 5-6
                                unified camera (its centre gives the view direction, one cache):
                                1 the unified camera's frustum and LOD filter the anchors for both eyes
                                (Eq. 6); 2 (GSC_STEREO_EXACT) the union of the two eyes' own filters,
                                each eye drawing only its own anchors, so that every eye's anchor
                                set is the per-eye method's; 0 off (per-eye derivation) */
  uint32_t cache_gaussians;  /* cache capacity in Gaussians per derivation view (0 = 4M) */
  uint32_t max_depth;        /* D_max of Alg. 1 (0 = 10) */
  uint32_t tile_w, tile_h;   /* blend tile in pixels (0 = 16 x 16): tile_w in {8, 16, 32}, tile_h a power of
                                two and a multiple of 128 / tile_w, 128 <= tile_w * tile_h <= 1024 */
  uint64_t pair_capacity;    /* initial (tile, Gaussian) pair capacity (0 = 16M); grows */
  float bg[3];               /* background colour */
  uint32_t use_graph;        /* 1: replay the frame's launch sequence as a CUDA graph */
  uint32_t flags;            /* GSC_FLAG_* */
  uint32_t blocks_per_sm;    /* blend: 0 = one block per tile; n = persistent grid of n blocks per SM
                                taking the tiles of all cameras from one counter */
  uint32_t out_format;       /* gsc_out_format of the images */
  uint32_t depth_guide;      /* gsc_depth_guide of the depth reuse form */
  uint32_t reserved[5];
} gsc_config;

/* Model description: host pointers, float32, row-major.  Copied by
 * gsc_load_model; the caller keeps ownership.  World units are metres. */
typedef struct {
  uint32_t n_anchors;
  uint32_t feat_dim;         /* must be 32 */
  uint32_t k;                /* must be 10 */
  uint32_t hidden;           /* must be 32 */
  uint32_t n_levels;         /* LOD levels (1 = LOD off) */
  float lod_dmax;            /* level l >= 1 drawn iff distance <= lod_dmax * 2^-l */
  const float* pos;          /* [N][3] anchor positions */
  const float* feat;         /* [N][32] anchor features */
  const float* offset;       /* [N][k][3] Gaussian offsets: mu_j = pos + offset_j */
  const float* scale;        /* [N] anchor scale s_a */
  const uint8_t* level;      /* [N] LOD level, 0 = coarsest */
  const float* W1[3];        /* per head [35][32], input = [feature(32), view dir(3)] */
  const float* b1[3];        /* per head [32] */
  const float* W2[3];        /* per head [32][out_h], out_h = k, 3k, 7k */
  const float* b2[3];        /* per head [out_h] */
  /* Octree-GS level selection (Sec. 2: the octree's levels of detail chosen
   * by distance).  Optional; NULL / 0 keep the plain distance rule above.
   * level_offset: [N] learned per-anchor level offsets Delta_a, finite,
   *   |Delta_a| <= 8.  An anchor of level l >= 1 is drawn iff
   *   l <= log2(lod_dmax / d) + Delta_a, i.e. d <= r_a with the float32
   *   radius r_a = (float)ldexp((double)lod_dmax * exp2((double)Delta_a), -l),
   *   evaluated once at load in float64 (so the decision is a float32
   *   comparison d^2 <= r_a^2, taken in the same order as the plain rule).
   * lod_blend: beta >= 0, in levels.  beta > 0 fades in an anchor of level
   *   l >= 1 as the camera approaches: its Gaussians' opacities are scaled by
   *   w = min(1, u / beta), u = log2(r_a / d) >= 0 (its margin in levels
   *   inside the switching distance; d^2 is the culling test's float32
   *   squared distance), so an anchor does not pop in when its level is
   *   switched on.  Applied after derivation and the cache. */
  const float* level_offset;
  float lod_blend;
  uint32_t reserved0;
} gsc_model_desc;

/* Pinhole camera: camera coords c = R x + t (x right, y down, z forward),
 * pixel (i, j) has its centre at (i + 0.5, j + 0.5). */
typedef struct {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  uint32_t width, height;
  float znear;
  int32_t stereo_partner;    /* index of the other eye in the same gsc_set_cameras call, or -1 */
  uint32_t model_id;         /* from gsc_load_model */
  uint32_t viewer;           /* cache owner: cameras of one viewer share its derivation cache */
} gsc_camera;

typedef struct {
  uint64_t visible_anchors;  /* summed over derivation views */
  uint64_t derived_anchors;  /* anchors decoded by the MLPs this frame (cache misses) */
  uint64_t records;          /* (Gaussian, camera) records projected */
  uint64_t valid_records;    /* records that cover at least one tile */
  uint64_t pairs;            /* (tile, Gaussian) pairs sorted and blended */
  uint32_t cache_depth;      /* reuse depth chosen for the next frame (viewer 0) */
  uint32_t error_flags;      /* bit 0 pair overflow, bit 1 wait timeout, bit 2 cache full */
  float ms_stage[8];         /* with GSC_FLAG_TIMING: cull, derive, sort1, scan+keygen, sort2, ranges, blend, total */
} gsc_frame_stats;

/* Fill *cfg with the defaults (stereo 2K, FP32, no reuse, 16x16 tiles, graph on). */
GSC_API void gsc_default_config(gsc_config* cfg);

/* Create a context on the current CUDA device.  cuda_stream is a cudaStream_t
 * (may be NULL).  Returns GSC_ERR_INVALID_ARG for bad config values,
 * GSC_ERR_OOM / GSC_ERR_CUDA on allocation failure (no context is returned). */
GSC_API int gsc_create(gsc_ctx** out, const gsc_config* cfg, void* cuda_stream);

/* Upload a model (Sec. 3.1 structured anchors; Eq. 3 decoder weights).
 * Validates the description (null pointers, dims, NaN positions are
 * rejected) and copies it into device memory; *model_id_out receives the id
 * used by gsc_camera.model_id.  Synchronous with respect to the host buffers. */
GSC_API int gsc_load_model(gsc_ctx* ctx, const gsc_model_desc* desc, uint32_t* model_id_out);

/* Set the cameras of the next frames (host array of n <= max_views).  Stereo
 * partners must reference each other, share intrinsics and model.  The
 * values are copied; the library uploads them with the frame. */
GSC_API int gsc_set_cameras(gsc_ctx* ctx, const gsc_camera* cams, uint32_t n);

/* Render one frame: out_rgb[i] is a caller-owned DEVICE pointer to a float32
 * [height][width][3] image for camera i.  With stats != NULL the call waits
 * for the frame, grows the pair buffer and re-renders if it overflowed, and
 * fills *stats.  With stats == NULL the call only enqueues work; a buffer
 * overflow or a wait timeout of any such frame since the last synchronising
 * call is reported by the next synchronising call (a render with stats,
 * gsc_synchronize): GSC_ERR_TIMEOUT, or GSC_ERR_CAPACITY after the buffers
 * have been grown to what those frames asked for.  The images of such a
 * frame are then invalid; render it again. */
GSC_API int gsc_render_frame(gsc_ctx* ctx, void* const* out_rgb, gsc_frame_stats* stats);

/* Same as gsc_render_frame, but out_rgb[i] are HOST pointers (pinned or
 * pageable); the device->host copies are part of the call, which returns
 * when the images are in host memory. */
GSC_API int gsc_render_frame_host(gsc_ctx* ctx, void* const* out_rgb, gsc_frame_stats* stats);

/* Pipelined host rendering for a stream of frames: enqueues the frame and
 * the copy of its images into out[i] (HOST pointers, pinned for the copy to
 * overlap, valid until gsc_wait_host returns) and returns at once.  The
 * device renders into one of two internal image sets while the previous
 * frame's images are still being copied to the host on a copy stream, so a
 * frame costs max(render, copy) rather than their sum.  The images of a
 * frame are complete when gsc_wait_host returns (or after two more frames
 * have been enqueued).  Buffer growth cannot re-render an asynchronous
 * frame: run one synchronous frame first; a later overflow or timeout is
 * reported by gsc_wait_host (GSC_ERR_CAPACITY / GSC_ERR_TIMEOUT, the
 * affected images invalid). */
GSC_API int gsc_render_frame_host_async(gsc_ctx* ctx, void* const* out);

/* Wait for all pipelined host frames; returns the first deferred error. */
GSC_API int gsc_wait_host(gsc_ctx* ctx);

/* Change the blend tiling of a context in place (models and cameras stay):
 * tile_w x tile_h as for gsc_config, blocks_per_sm as for gsc_config.  Used
 * by the autotuner (Sec. 4 renders eyes "independently or in batching"; the
 * tile shape and grid of the batched frame are picked by timing).  Invalid
 * values return GSC_ERR_INVALID_ARG and leave the tiling unchanged. */
GSC_API int gsc_set_tiling(gsc_ctx* ctx, uint32_t tile_w, uint32_t tile_h, uint32_t blocks_per_sm);

/* ---- learned reuse predictor -------------------------------------------
 * An extension of the cache of Sec. 4 (the paper reuses by the depth rule of
 * Alg. 1 / Eq. 4 only): with reuse = GSC_REUSE_LEARNED a valid line (age <=
 * D_max) is reused iff p = sigmoid(w2 . relu(W1^T z + b1) + b2) >= 0.5, else
 * the anchor is decoded again.  z (36 floats): the anchor feature (32),
 * 1024 x the change of the unit direction from the derivation camera centre
 * to the anchor since the line was decoded (3), and plog2(distance) - 8 (1),
 * plog2(m 2^e) = e + (m - 1), m in [1, 2).  The decision uses float32 in a
 * fixed operation order with bfloat16-rounded weights.  Parameters are a
 * flat float array: W1 [36][64] input-major, b1 [64], w2 [64], b2 [1]. */
#define GSC_REUSE_NPARAM 2433

/* Set the predictor's float32 master weights (host array of n_params =
 * GSC_REUSE_NPARAM finite floats, copied).  Required before rendering in
 * the learned form and before training. */
GSC_API int gsc_reuse_set_weights(gsc_ctx* ctx, const float* params, uint32_t n_params);

/* Copy the float32 master weights (e.g. after gsc_reuse_train) to params. */
GSC_API int gsc_reuse_get_weights(gsc_ctx* ctx, float* params, uint32_t n_params);

/* Training samples of the last frame (context created with
 * GSC_FLAG_REUSE_COLLECT and a reuse form): for derivation view dview, one
 * sample per visible anchor that held a valid line before the frame, in
 * visible order: z [n][36], label (1: reusing the line keeps every kept
 * Gaussian's opacity and opacity-weighted colour within 1/255 of a fresh
 * decode of this frame, and the same Gaussians kept; 0 otherwise) and the
 * anchor's index in the view's visible list.  Any output may be NULL; *n
 * receives the number of samples, at most cap are written.  Host memory. */
GSC_API int gsc_reuse_collect(gsc_ctx* ctx, uint32_t dview, float* z, uint8_t* label, uint32_t* vis_index,
                              uint64_t cap, uint64_t* n);

/* Train the predictor on the GPU from the current weights: n samples
 * (z [n][36] float, label [n] 0/1, host memory), `epochs` passes in
 * mini-batches of `batch`, Adam with step size lr (beta1 0.9, beta2 0.999,
 * eps 1e-8) on float32 master weights, forward/backward with their bfloat16
 * rounding, mean binary cross-entropy.  order: epochs x n sample indices
 * (host), or NULL for a shuffle per epoch drawn from SplitMix64(seed).
 * epoch_loss (may be NULL) receives the mean loss of each epoch.  The
 * trained weights replace the context's; the Adam state starts from zero. */
GSC_API int gsc_reuse_train(gsc_ctx* ctx, const float* z, const uint8_t* label, uint64_t n, uint32_t epochs,
                            uint32_t batch, float lr, uint64_t seed, const uint32_t* order, float* epoch_loss);

/* Empty every derivation cache (Sec. 4): the next frame decodes all anchors. */
GSC_API int gsc_cache_reset(gsc_ctx* ctx);

/* Wait for all enqueued frames and report deferred errors. */
GSC_API int gsc_synchronize(gsc_ctx* ctx);

/* Message of the last error of ctx (never NULL; "" after success). */
GSC_API const char* gsc_last_error(const gsc_ctx* ctx);

/* Free the context and all its device memory (waits for its stream). */
GSC_API void gsc_destroy(gsc_ctx* ctx);

GSC_API int gsc_version(void);

/* Largest n accepted by gsc_scan_u32_noalloc. */
#define GSC_NOALLOC_SCAN_MAX_N (1u << 24)

/* Exclusive prefix sum of n uint32 values for callers that cannot allocate
 * device memory: a frame loop under a real-time budget (an allocation can
 * synchronise the device and stall the frame) or a host application whose
 * pool owns every device allocation and that hands plug-ins only the
 * buffers they work on.  The paper has no counterpart to this call; it is a
 * service of the library, built on the same decoupled look-back scan the
 * renderer uses for its pair offsets.
 *   d_in    device pointer, n uint32 values (read only)
 *   d_out   device pointer, n uint32 results: d_out[i] = sum of d_in[0..i-1];
 *           may equal d_in (in place)
 *   n       0 .. GSC_NOALLOC_SCAN_MAX_N (16,777,216); larger n returns
 *           GSC_ERR_INVALID_ARG before any work is enqueued
 *   d_total device pointer to one uint32 receiving the sum, or NULL
 *   cuda_stream  cudaStream_t to run on (NULL = legacy default stream)
 * The call allocates nothing: its working memory is a fixed 32,800-byte
 * device array inside the library, present on every GPU that loads the
 * library until the process exits.  Every call looks that array's address
 * up (cudaGetSymbolAddress) for the device and context current at the call;
 * no address is kept between calls.  The call reads an error word back and
 * synchronises the stream, so it must not be made on a stream that is being
 * captured into a CUDA graph: such a call returns GSC_ERR_INVALID_ARG and
 * enqueues nothing.  Calls whose work overlaps on the GPU (other threads or
 * streams) share the array and race: serialise them.  The call is
 * synchronous: it returns after the scan has finished on the stream.
 * Returns GSC_OK; GSC_ERR_INVALID_ARG for bad pointers or n, for a
 * capturing stream, or when the sum of the inputs reaches 2^30;
 * GSC_ERR_TIMEOUT if a bounded device-side wait gave up; GSC_ERR_CUDA if a
 * CUDA call failed.  After GSC_ERR_INVALID_ARG for the sum and after
 * GSC_ERR_TIMEOUT the contents of d_out and *d_total are unspecified; the
 * next call starts from a cleared error word. */
GSC_API int gsc_scan_u32_noalloc(const uint32_t* d_in, uint32_t* d_out, uint64_t n, uint32_t* d_total,
                                 void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* GSC_H */
