/*
 * gsc_debug.h - test-only exports of the GS-Cache frame renderer.
 *
 * These read back the intermediate buffers of the LAST rendered frame so that
 * each stage can be compared with an independent reference on its own.  All
 * are synchronous (they wait for the context's stream) and copy into
 * caller-owned HOST memory.  For each: pass cap = capacity of the output
 * arrays in elements of the stated unit; *n receives the number available;
 * nothing is written past cap.  Return values are gsc_status codes.
 */
#ifndef GSC_DEBUG_H
#define GSC_DEBUG_H

#include "gsc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Visible anchor ids (ascending) of derivation view d (anchor filtering,
 * Sec. 3.2).  Derivation views are the cameras in order, except that with
 * stereo_unify each stereo pair forms one view at the position of its
 * lower-indexed camera.  Unit: uint32 ids. */
GSC_API int gsc_debug_visible(gsc_ctx* ctx, uint32_t d, uint32_t* ids, uint64_t cap, uint64_t* n);

/* Exact stereo form (stereo_unify = GSC_STEREO_EXACT): for derivation view
 * d's visible anchors (as gsc_debug_visible), a mask of the cameras whose
 * own filter keeps each (bit 0: the pair's lower-indexed camera, bit 1: the
 * other).  Only meaningful for exact stereo views.  Unit: uint8 masks. */
GSC_API int gsc_debug_visible_eyes(gsc_ctx* ctx, uint32_t d, uint8_t* eyes, uint64_t cap, uint64_t* n);

/* Number of derivation views of the last frame and the camera each feeds. */
GSC_API int gsc_debug_dviews(gsc_ctx* ctx, uint32_t* n_dviews, int32_t* first_cam /* [GSC_MAX_VIEWS] */);

/* Derived attributes (Eq. 3) of derivation view d, needs GSC_FLAG_DEBUG_ATTRS:
 * per visible anchor i and Gaussian j, 11 floats: alpha, colour(3),
 * scale(3), quaternion(4) (w,x,y,z).  Unit: anchors ([n][k][11] floats). */
GSC_API int gsc_debug_attrs(gsc_ctx* ctx, uint32_t d, float* attrs, uint64_t cap, uint64_t* n);

/* Projected records, one per (camera, visible anchor, Gaussian), record
 * index r = base(camera) + i*k + j.  Per record 12 floats: mean x, mean y,
 * conic A, B, C (q = A dx^2 + 2 B dx dy + C dy^2), opacity, tau (coverage
 * threshold on q), depth, colour(3), and the bits of a uint32 word
 * (camera index in bits 0-15, bit 31 = record passed the projection tests);
 * plus the sort key (depth bits, 0xFFFFFFFF when unused) and tile count.
 * A record that covers no tile is reported as zeros with its camera index
 * and a tile count of 0 (the device keeps only its key).  Unit: records. */
GSC_API int gsc_debug_records(gsc_ctx* ctx, float* rec12, uint32_t* depth_key, uint32_t* tile_count,
                      uint64_t cap, uint64_t* n);

/* Sorted (key, value) pairs: key = tile_base(camera) + tile, value = record.
 * Unit: pairs. */
GSC_API int gsc_debug_pairs(gsc_ctx* ctx, uint32_t* keys, uint32_t* vals, uint64_t cap, uint64_t* n);

/* Records in depth order after the first sort (values only).  Unit: records. */
GSC_API int gsc_debug_depth_order(gsc_ctx* ctx, uint32_t* vals, uint64_t cap, uint64_t* n);

/* Tile ranges [start, end) into the sorted pairs, for every tile of every
 * camera in key order.  Unit: tiles ([n][2] uint32). */
GSC_API int gsc_debug_ranges(gsc_ctx* ctx, uint32_t* ranges, uint64_t cap, uint64_t* n);

/* Final transmittance of camera v, needs GSC_FLAG_DEBUG_T.  Unit: pixels. */
GSC_API int gsc_debug_final_T(gsc_ctx* ctx, uint32_t v, float* T, uint64_t cap, uint64_t* n);

/* Cache of derivation view d in the reuse forms (Sec. 4, Alg. 1): per visible
 * anchor of the last frame its line status (line index | 0x80000000 for a
 * reuse, the line index for a decode into a line, 0x7FFFFFFF for a decode
 * without a line), and 8 state words: frame counter, depth for the next
 * frame, misses, new anchors, free lines, visible anchors, D_max, lines.
 * Unit: visible anchors. */
GSC_API int gsc_debug_cache(gsc_ctx* ctx, uint32_t d, uint32_t* vstat, uint64_t cap, uint64_t* n, uint32_t* state8);

/* Upper bound on the polls of every bounded device-side wait (0 makes any
 * wait that does not succeed at once give up).  Default 1 << 20. */
GSC_API int gsc_debug_set_spin_limit(gsc_ctx* ctx, uint32_t limit);

/* Standalone radix sort of n (key, value) pairs in host memory through the
 * library's sort kernels (keys sorted on bits [0, bits), stable).  For
 * testing the sort against a library sort.  Unit: pairs. */
GSC_API int gsc_debug_sort_pairs(gsc_ctx* ctx, uint32_t* keys, uint32_t* vals, uint64_t n, uint32_t bits);

/* Timeout path: runs a kernel whose bounded wait targets a word that no
 * kernel writes, with the given poll limit.  Returns GSC_ERR_TIMEOUT when the
 * wait gave up and reported it (the expected outcome); the context stays
 * usable. */
GSC_API int gsc_debug_wait_timeout(gsc_ctx* ctx, uint32_t spin_limit);

/* Standalone exclusive scan of n uint32 values in host memory through the
 * library's decoupled look-back scan kernel; *total receives the sum. */
GSC_API int gsc_debug_scan(gsc_ctx* ctx, uint32_t* vals, uint64_t n, uint64_t* total);

/* Bytes of the per-frame description uploaded host -> device by every
 * render call (cameras with their constants, output pointers). */
GSC_API int gsc_debug_frame_upload_bytes(void);

/* Gradient of the predictor's mean binary cross-entropy over n samples (host
 * z [n][36], label [n]) at the current weights (bfloat16-rounded, as in
 * training), one forward/backward through the training kernels: grad
 * [GSC_REUSE_NPARAM] and *loss (may be NULL), host memory. */
GSC_API int gsc_debug_reuse_grad(gsc_ctx* ctx, const float* z, const uint8_t* label, uint64_t n, float* grad,
                                 float* loss);

/* Blend work of the last rendered frame, needs GSC_FLAG_BLEND_WORK (host
 * work[2]): work[0] = (pixel, Gaussian) evaluations of the front-to-back
 * walk of every pixel - each Gaussian of its tile's list up to and including
 * the one at which the pixel stops (T would fall below 1e-4), or all of
 * them; work[1] = pixel evaluations the blend issued: 4 per lane of each
 * warp for every Gaussian whose opacity-aware box meets the warp's rows
 * (each one exp2, whether or not its pixel still blends).  Synchronises. */
GSC_API int gsc_debug_blend_work(gsc_ctx* ctx, uint64_t* work);

/* Measured throughput of the current device's arithmetic units (host
 * rates[3], per second): [0] exp2 results (ex2.approx, the special function
 * unit), [1] FP32 FMA lane operations (scalar), [2] FP32 FMA lane operations
 * of the packed FP32x2 form (two per instruction).  Runs three short probe
 * kernels (a few ms) on a stream of its own; allocates and frees a small
 * buffer.  Returns GSC_ERR_CUDA / GSC_ERR_OOM on failure. */
GSC_API int gsc_debug_pipe_rates(double* rates);

#ifdef __cplusplus
}
#endif
#endif /* GSC_DEBUG_H */
