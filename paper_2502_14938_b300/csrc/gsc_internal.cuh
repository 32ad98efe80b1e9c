// Internal device-side definitions of the GS-Cache frame renderer (sm_103a).
//
// Frame data flow (all sizes live in device memory, so one frame is a fixed
// launch sequence that can be replayed as a CUDA graph without host reads):
//   frame_begin  -> per-camera constants, unified cameras (Eq. 5-6), counters
//   cull         -> ascending visible anchor ids per derivation view (K1)
//   plan         -> record bases per camera
//   derive       -> MLP decode (Eq. 3) fused with EWA projection and exact
//                   tile counting (Eq. 1-2, Sec. 6): one record per
//                   (camera, anchor, Gaussian)
//   sort #1      -> records in depth order (32-bit depth key, invalid dropped)
//   scan+keygen  -> (tile key, record) pairs in depth order
//   sort #2      -> stable sort by tile key => (tile, depth, Gaussian id)
//   ranges+blend -> per-tile front-to-back alpha blending
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "gsc.h"

namespace gsc {

constexpr int K = GSC_K;            // Gaussians per anchor
constexpr int FDIM = GSC_FEAT_DIM;  // anchor feature width
constexpr int HID = GSC_HIDDEN;     // hidden width of each head
constexpr int IN = FDIM + 3;        // MLP input: feature + unit view direction
constexpr int NH = 3 * HID;         // concatenated hidden width of the 3 heads
constexpr int NOUT = K + 3 * K + 7 * K;  // 110 head outputs
constexpr int MAXV = GSC_MAX_VIEWS;
constexpr int MAX_MODELS = 8;
constexpr int REC_F4 = 3;           // float4s per record

// packed float32 weights: W1cat [IN][NH], b1cat [NH], W2T [NOUT][HID], b2cat [NOUT]
constexpr int WOFF_W1 = 0;
constexpr int WOFF_B1 = WOFF_W1 + IN * NH;
constexpr int WOFF_W2T = WOFF_B1 + NH;
constexpr int WOFF_B2 = WOFF_W2T + NOUT * HID;
constexpr int W_FLOATS = WOFF_B2 + NOUT;

enum : uint32_t { ERR_PAIR_OVERFLOW = 1u, ERR_TIMEOUT = 2u, ERR_CACHE_FULL = 4u, ERR_REC_OVERFLOW = 8u,
                  ERR_BOUNDS = 16u };

// Stores whose index comes from data (compaction offsets, sort ranks, cache
// lines, list cursors) are written as `if (GSC_IN_BOUNDS(i, cap, err)) p[i] =
// v;`.  The bounds-checked build of the library (GSC_DEBUG_BOUNDS, the
// substitute for a memory checker) tests i < cap there, and on a miss sets
// ERR_BOUNDS in *err and skips the store; the normal build stores
// unconditionally.
#ifdef GSC_DEBUG_BOUNDS
#define GSC_IN_BOUNDS(i, cap, err) \
  ((uint64_t)(i) < (uint64_t)(cap) ? true : (atomicOr((err), (uint32_t)ERR_BOUNDS), false))
#else
#define GSC_IN_BOUNDS(i, cap, err) true
#endif

constexpr uint32_t INVALID_KEY = 0xFFFFFFFFu;
constexpr uint32_t REC_VALID_BIT = 0x80000000u;

struct CamDev {  // camera with derived constants (prepared by the library's host code each frame)
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  int32_t W, H;
  float znear;
  float pc[3];     // centre -R^T t (float64 then rounded)
  float pc_lo[3];  // float64 centre - pc: (pc, pc_lo) is a double-float centre
  float dt[3];     // t + R pc in float64: what R (x - pc) misses of R x + t when the
                   // float32 R is not exactly orthonormal (|dt| ~ 1e-7 |t|)
  float gx, gy;    // 1.3 * (0.5 W / fx), 1.3 * (0.5 H / fy) in float32
  int32_t ntx, nty;
  uint32_t tile_base;
  int32_t model;
};

struct FrameIn {  // host -> device per frame
  uint32_t n_cams, n_dviews;
  uint32_t tile_w, tile_h;
  uint32_t spin_limit;
  uint32_t total_tiles, tile_bits;
  uint32_t out_format;               // gsc_out_format
  uint32_t keep_err;                 // 1: OR the frame's error bits into err_sticky (frames nobody waits for)
  uint32_t cap_vis;                  // capacities of the frame's buffers (the bounds-checked build's
  uint32_t cap_rec;                  // limits): visible ids per view, records, pairs
  uint32_t cap_pairs;
  uint32_t depth_base;               // bits of the smallest near plane of the frame's cameras
  uint32_t pad[2];
  float bg[4];
  unsigned long long out_rgb[MAXV];  // float* [H][W][3] per camera (device)
  unsigned long long out_T[MAXV];    // float* [H][W] per camera or 0
  CamDev cam[MAXV];                  // cameras with their constants
  CamDev dcam[MAXV];                 // derivation views (unified camera of a stereo pair, Eq. 5-6)
  int32_t dview_of_cam[MAXV];
  int32_t dview_cam[MAXV][2];
  int32_t dview_exact[MAXV];         // 1: a stereo pair filtered by the union of its eyes' own filters
};

constexpr int DEPTH_HIST_WORDS = 3 * 512 + 256;

struct FrameDev {  // device-resident per-frame plan and counters
  uint32_t frame;               // frame counter, starts at 1 (epochs of look-back words)
  uint32_t n_cams, n_dviews;
  uint32_t tile_w, tile_h;
  uint32_t total_tiles, tile_bits;
  uint32_t spin_limit;
  uint32_t cap_vis, cap_rec, cap_pairs;  // buffer capacities (bounds-checked build)
  CamDev cam[MAXV];
  CamDev dcam[MAXV];
  int32_t dview_of_cam[MAXV];
  int32_t dview_cam[MAXV][2];   // cameras fed by a derivation view (-1 unused)
  int32_t dview_exact[MAXV];    // 1: the view's anchors are the union of its two cameras' own sets,
                                // with a per-anchor mask of the cameras that keep it (exact stereo form)
  // after culling
  uint32_t vis_count[MAXV];
  uint32_t item_base[MAXV + 1];  // prefix over derivation views of vis_count
  uint32_t rec_base[MAXV + 1];   // prefix over cameras of K * vis_count[dview]
  uint32_t n_items, n_records;
  // counters of the frame
  uint32_t n_valid;             // records with key != INVALID (set by sort #1 histogram)
  uint32_t n_pairs;             // pairs requested (may exceed capacity)
  uint32_t n_pairs_used;        // min(n_pairs, capacity)
  uint32_t err;
  uint32_t n_records_need;      // records the frame asked for (may exceed capacity)
  uint32_t n_big;               // records in the key generation's large-record list
  uint32_t n_derived;           // anchors decoded this frame (visible minus cache hits)
  uint32_t cache_depth;         // reuse depth of derivation view 0 for the next frame
  uint32_t ctr[64];             // dynamic tile counters of look-back kernels
  // digit histograms of the two sorts, accumulated by the kernels that
  // produce their keys: projection, the valid depth keys minus depth_base
  // (3 x 512 for the 9-bit digits, then 256 for bits 24-31); key
  // generation, the tile keys of the written pairs (4 x 256)
  alignas(16) uint32_t hist_depth[DEPTH_HIST_WORDS];
  alignas(16) uint32_t hist_tile[4 * 256];
  uint32_t depth_base;          // bits of the nearest near plane: every valid depth key is above it
  uint32_t depth_wide;          // 1: some valid depth key - depth_base needs more than 27 bits
  uint32_t err_sticky;          // error bits of all frames since the host last read them
  uint32_t need_sticky[2];      // largest records / pairs those frames asked for
  // blend work of the frame, counted only by the counting blend variant:
  // [0] (pixel, Gaussian) evaluations of the front-to-back walk (every
  //     Gaussian of the tile's list up to and including the one a pixel
  //     stops at), [1] pixel slots issued through the inner loop (4 per lane
  //     for each Gaussian whose box meets the warp's band; one exp2 each)
  unsigned long long blend_work[2];
};

struct ModelDev {
  uint32_t n, n_levels;
  float lod_dmax;
  float fp8_inv_sx;       // FP8 form: 1 / s_x (input scale, a power of two)
  const float* px;
  const float* py;
  const float* pz;
  const uint8_t* level;
  const float* lod_r;     // [N] Octree-GS switching radius (+inf at level 0), or null: plain distance rule
  float lod_beta;         // level fade width in levels (0: none; needs lod_r)
  const float4* feat;     // [N][8]
  const float* offs;      // [N][K][3]
  const float* scale;     // [N]
  const float* w32;       // packed weights, W_FLOATS
  const void* feat_bf16;  // [N][32] bf16 (tensor-core forms)
  const void* w_tc;       // tensor-core weight image, bf16 (65,536 bytes)
  const void* feat_fp8;   // [N][32] e4m3 of feature / s_x (FP8 form)
  const void* w_tc8;      // tensor-core weight image, two-term e4m3 + scales (70,016 bytes)
};

// One derivation view's cache of derived Gaussians (Sec. 4).
// CS_HW: lines at or above it have never held an anchor this cache's life
// (assignment takes free lines in ascending order, so used lines stay below
// it); the probe and the scan cover lines [0, CS_HW) only.  CS_HW_NEXT: the
// value for the next frame, written by the assignment, taken at the tick.
enum : int { CS_T = 0, CS_DEPTH, CS_MISSES, CS_NEW, CS_FREE, CS_VIS, CS_DMAX, CS_S, CS_SCAN_N, CS_SCAN_TOT, CS_GUIDE,
             CS_HW, CS_HW_NEXT, CS_WORDS };
constexpr uint32_t LINE_HIT = 0x80000000u;   // vstat: the anchor reuses its line
constexpr uint32_t LINE_NONE = 0x7FFFFFFFu;  // vstat: decoded without a line
struct CacheDev {
  uint32_t* slot_of;      // [N of the model] line of an anchor (0xFFFFFFFF none)
  uint32_t* slot_anchor;  // [S] anchor of a line (0xFFFFFFFF unused)
  uint32_t* slot_frame;   // [S] frame of the line's last decode
  uint2* slot_attr;       // [S][K][3]: 12 float16 per Gaussian (alpha, c, s, q, 0)
  uint32_t* vstat;        // [visible] line | LINE_HIT, or LINE_NONE
  uint32_t* flags;        // [hw + visible]: line is free (lines below CS_HW), then visible anchor is new
  uint32_t* ranks;        // [hw + visible]: exclusive prefix of flags (one scan)
  uint32_t* free_list;    // [S] free lines below CS_HW in ascending order
  uint32_t* miss;         // [visible] visible indices to decode
  uint32_t* state;        // [CS_WORDS]
  float4* slot_dir;       // [S] unit direction camera -> anchor when the line was decoded
  float* cz;              // [visible][36] predictor inputs of the frame (collection)
  uint8_t* clab;          // [visible] label: 1 reuse ok, 0 not, 255 no valid line (collection)
  uint32_t S;
  uint32_t active;
};

// Depth-rule probe of visible anchor vi (anchor a) of a view's cache (Alg. 1,
// Eq. 4's reuse depth): hit = a valid line decoded at most `depth` frames
// ago; lines older than D are invalid.  Writes the line status and the
// anchor's new flag (at hw + vi) and appends a miss to the decoder's list
// (bounded by miss_cap).  Used by the cache probe kernel and by the cull's
// write pass, which probes each id as it writes it.
__device__ __forceinline__ void cache_probe_depth(const CacheDev& cd, uint32_t a, uint32_t vi, uint32_t t,
                                                  uint32_t depth, uint32_t D, uint32_t hw, uint32_t miss_cap,
                                                  uint32_t* err) {
  const uint32_t s = cd.slot_of[a];
  bool valid = s < cd.S && cd.slot_anchor[s] == a;
  const uint32_t age = valid ? t - cd.slot_frame[s] : 0xFFFFFFFFu;
  valid = valid && age <= D;
  const bool hit = valid && age <= depth;
  cd.vstat[vi] = hit ? (s | LINE_HIT) : (valid ? s : LINE_NONE);
  cd.flags[hw + vi] = valid ? 0u : 1u;
  if (!hit) {
    const uint32_t mi = atomicAdd(&cd.state[CS_MISSES], 1u);
    if (GSC_IN_BOUNDS(mi, miss_cap, err)) cd.miss[mi] = vi;
  }
}
// Free flag of line s (unused, or past D_max) for the scan of free lines.
__device__ __forceinline__ uint32_t cache_line_free(const CacheDev& cd, uint32_t s, uint32_t t, uint32_t D) {
  return (cd.slot_anchor[s] == 0xFFFFFFFFu || t - cd.slot_frame[s] > D) ? 1u : 0u;
}

struct Records {
  float4* geo;    // mean x, mean y, A, B
  float4* cop;    // C, opacity, tau_cov, depth
  float4* col;    // r, g, b, bits(view | valid bit)
  float4* aux;    // for the blend: C, log2(opacity), box half-width, box half-height
  uint32_t* key;  // depth bits or INVALID_KEY
  uint32_t* cnt;  // covered tiles
};

// ----------------------------------------------------------------- look-back words
// 64-bit status word: [63:32] epoch, [31:30] flag (1 aggregate, 2 inclusive prefix), [29:0] value
__device__ __forceinline__ unsigned long long lb_pack(uint32_t epoch, uint32_t flag, uint32_t v) {
  return ((unsigned long long)epoch << 32) | ((unsigned long long)flag << 30) | (unsigned long long)(v & 0x3FFFFFFFu);
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Exclusive prefix of tile t from its predecessors' words (stride apart),
// polling at most spin_limit times in total; on timeout sets ERR_TIMEOUT and
// returns what it has (the frame is then reported invalid).  Once any wait
// of the launch has timed out, the others give up at their next check, so
// a failure costs one timeout, not one per tile.  The partial prefix is
// never larger than the true one, so the writes it steers stay in bounds.
// One thread per chain; LB_AHEAD predecessor words are loaded at once so a
// walk over aggregates costs one memory round trip per LB_AHEAD tiles.
constexpr int LB_AHEAD = 8;
__device__ __forceinline__ uint32_t lb_exclusive(const unsigned long long* words, uint32_t stride, uint32_t t,
                                                 uint32_t epoch, uint32_t spin_limit, uint32_t* err) {
  uint32_t excl = 0;
  int j = (int)t - 1;
  uint32_t spins = 0;
  while (j >= 0) {
    unsigned long long w[LB_AHEAD];
#pragma unroll
    for (int u = 0; u < LB_AHEAD; ++u) w[u] = j - u >= 0 ? ld_relaxed_u64(words + (size_t)(j - u) * stride) : 0ull;
    int used = 0;
    bool done = false, stalled = false;
#pragma unroll
    for (int u = 0; u < LB_AHEAD; ++u) {
      if (done || stalled || j - u < 0) continue;
      const uint32_t ep = (uint32_t)(w[u] >> 32);
      const uint32_t flag = (uint32_t)(w[u] >> 30) & 3u;
      if (ep != epoch || flag == 0) {
        stalled = true;
        continue;
      }
      excl += (uint32_t)(w[u] & 0x3FFFFFFFu);
      ++used;
      done = flag == 2;
    }
    if (done) break;
    j -= used;
    if (stalled) {
      if (++spins > spin_limit) {
        atomicOr(err, ERR_TIMEOUT);
        break;
      }
      if ((spins & 255u) == 0 && (*(volatile uint32_t*)err & ERR_TIMEOUT)) break;
      __nanosleep(32);
    }
  }
  return excl;
}

// The same for one chain walked by a whole warp (all 32 lanes call it, the
// result is returned in every lane): lane l reads predecessor j - l, so a
// window of 32 words costs one round trip; the window is consumed up to the
// first word that is not ready or through the first inclusive one.
__device__ __forceinline__ uint32_t lb_exclusive_warp(const unsigned long long* words, uint32_t stride, uint32_t t,
                                                      uint32_t epoch, uint32_t spin_limit, uint32_t* err) {
  const int lane = (int)(threadIdx.x & 31u);
  uint32_t excl = 0;
  int j = (int)t - 1;
  uint32_t spins = 0;
  while (j >= 0) {
    const int k = j - lane;
    const unsigned long long w = k >= 0 ? ld_relaxed_u64(words + (size_t)k * stride) : lb_pack(epoch, 2u, 0u);
    const uint32_t flag = (uint32_t)(w >> 30) & 3u;
    const bool ready = (uint32_t)(w >> 32) == epoch && flag != 0;
    const unsigned not_ready = __ballot_sync(0xffffffffu, !ready);
    const unsigned incl = __ballot_sync(0xffffffffu, ready && flag == 2);
    const int first_nr = not_ready ? __ffs(not_ready) - 1 : 32;
    const int first_inc = incl ? __ffs(incl) - 1 : 32;
    const int take = first_inc < first_nr ? first_inc + 1 : first_nr;  // lanes [0, take) are summed
    uint32_t v = lane < take ? (uint32_t)(w & 0x3FFFFFFFu) : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    excl += v;
    if (first_inc < first_nr) break;
    j -= take;
    if (take == 0) {
      if (++spins > spin_limit) {
        if (lane == 0) atomicOr(err, ERR_TIMEOUT);
        break;
      }
      if ((spins & 255u) == 0 && (*(volatile uint32_t*)err & ERR_TIMEOUT)) break;
      __nanosleep(32);
    }
  }
  return excl;
}

// ----------------------------------------------------------------- small helpers
__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

template <int NT>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* s_warp, uint32_t* total) {
  // s_warp: NT/32 + 1 words of shared memory
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t s = (lane < (uint32_t)(NT / 32)) ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= (uint32_t)o) s += y;
    }
    if (lane < (uint32_t)(NT / 32)) s_warp[lane] = s;  // inclusive per warp
    if (lane == (uint32_t)(NT / 32) - 1) s_warp[NT / 32] = s;
  }
  __syncthreads();
  uint32_t base = (w == 0) ? 0u : s_warp[w - 1];
  if (total) *total = s_warp[NT / 32];
  uint32_t r = base + x - v;
  __syncthreads();
  return r;
}

// Tiles covered by the ellipse q(D) = A Dx^2 + 2 B Dx Dy + C Dy^2 <= tau
// (opacity-aware extent, Sec. 6): a tile counts iff the hull of its pixel
// centres meets the ellipse.  Per tile row the restricted ellipse is convex,
// so its x-range comes from the closed-form extreme points
//   Dy* = -B sqrt(tau / (C det)),  x(Dy) = (-B Dy +- sqrt(A tau - det Dy^2)) / A.
// Every operation is a correctly rounded float32 op (no contraction), so the
// count pass and the emit pass agree exactly.  Tile sizes are powers of two,
// so x / TW is computed as x * (1/TW), which is the same correctly rounded
// value.  f(tile) is called per tile.
struct Cover {
  float mx, my, A, B, tau, det, ey, ys, fTW, rTW;
  int ntx, ty0, ty1;
};

// Rows [ty0, ty1] of tiles the ellipse can touch; false if it covers nothing.
__device__ __forceinline__ bool cover_setup(Cover& cv, float mx, float my, float A, float B, float C, float tau,
                                            int W, int H, int TW, int TH) {
  const float det = __fsub_rn(__fmul_rn(A, C), __fmul_rn(B, B));
  if (!(tau > 0.f) || !(det > 0.f) || !(A > 0.f) || !(C > 0.f)) return false;
  const int nty = (H + TH - 1) / TH;
  cv.ntx = (W + TW - 1) / TW;
  cv.mx = mx; cv.my = my; cv.A = A; cv.B = B; cv.tau = tau; cv.det = det;
  cv.ey = __fsqrt_rn(__fdiv_rn(__fmul_rn(tau, A), det));
  cv.ys = __fmul_rn(-B, __fsqrt_rn(__fdiv_rn(tau, __fmul_rn(C, det))));
  cv.fTW = (float)TW;
  cv.rTW = 1.0f / (float)TW;
  const float fTH = (float)TH, rTH = 1.0f / (float)TH;
  float fy0 = ceilf(__fmul_rn(__fsub_rn(__fsub_rn(my, cv.ey), __fsub_rn(fTH, 0.5f)), rTH));
  float fy1 = floorf(__fmul_rn(__fsub_rn(__fadd_rn(my, cv.ey), 0.5f), rTH));
  fy0 = fminf(fmaxf(fy0, 0.f), (float)nty);
  fy1 = fminf(fmaxf(fy1, -1.f), (float)(nty - 1));
  cv.ty0 = (int)fy0;
  cv.ty1 = (int)fy1;
  return cv.ty0 <= cv.ty1;
}

// Column range [tx0, tx1] of tile row ty (empty when tx0 > tx1).
__device__ __forceinline__ void cover_row(const Cover& cv, int ty, int TH, int& tx0, int& tx1) {
  float b0 = __fsub_rn(__fadd_rn((float)(ty * TH), 0.5f), cv.my);
  float b1 = __fsub_rn(__fsub_rn((float)(ty * TH + TH), 0.5f), cv.my);
  b0 = fmaxf(b0, -cv.ey);
  b1 = fminf(b1, cv.ey);
  if (b0 > b1) {
    tx0 = 1;
    tx1 = 0;
    return;
  }
  const float yr = fminf(fmaxf(cv.ys, b0), b1);
  const float yl = fminf(fmaxf(-cv.ys, b0), b1);
  const float dr = __fsub_rn(__fmul_rn(cv.A, cv.tau), __fmul_rn(cv.det, __fmul_rn(yr, yr)));
  const float dl = __fsub_rn(__fmul_rn(cv.A, cv.tau), __fmul_rn(cv.det, __fmul_rn(yl, yl)));
  const float xr = __fdiv_rn(__fadd_rn(__fmul_rn(-cv.B, yr), __fsqrt_rn(fmaxf(dr, 0.f))), cv.A);
  const float xl = __fdiv_rn(__fsub_rn(__fmul_rn(-cv.B, yl), __fsqrt_rn(fmaxf(dl, 0.f))), cv.A);
  float fx0 = ceilf(__fmul_rn(__fsub_rn(__fadd_rn(cv.mx, xl), __fsub_rn(cv.fTW, 0.5f)), cv.rTW));
  float fx1 = floorf(__fmul_rn(__fsub_rn(__fadd_rn(cv.mx, xr), 0.5f), cv.rTW));
  fx0 = fminf(fmaxf(fx0, 0.f), (float)cv.ntx);
  fx1 = fminf(fmaxf(fx1, -1.f), (float)(cv.ntx - 1));
  tx0 = (int)fx0;
  tx1 = (int)fx1;
}

template <typename Fn>
__device__ __forceinline__ void cover_tiles_f32(float mx, float my, float A, float B, float C, float tau,
                                                int W, int H, int TW, int TH, Fn f) {
  Cover cv;
  if (!cover_setup(cv, mx, my, A, B, C, tau, W, H, TW, TH)) return;
  for (int ty = cv.ty0; ty <= cv.ty1; ++ty) {
    int tx0, tx1;
    cover_row(cv, ty, TH, tx0, tx1);
    for (int tx = tx0; tx <= tx1; ++tx) f(ty * cv.ntx + tx);
  }
}

// Number of covered tiles (same arithmetic as cover_tiles_f32).
__device__ __forceinline__ uint32_t cover_count_f32(float mx, float my, float A, float B, float C, float tau, int W,
                                                    int H, int TW, int TH) {
  Cover cv;
  if (!cover_setup(cv, mx, my, A, B, C, tau, W, H, TW, TH)) return 0;
  uint32_t n = 0;
  for (int ty = cv.ty0; ty <= cv.ty1; ++ty) {
    int tx0, tx1;
    cover_row(cv, ty, TH, tx0, tx1);
    if (tx1 >= tx0) n += (uint32_t)(tx1 - tx0 + 1);
  }
  return n;
}

// ----------------------------------------------------------------- launchers (host)
struct SortBufs {
  uint32_t* hist;                 // [4][256] global digit counts
  unsigned long long* status;     // look-back words [tiles][256]
};

// counter / epoch slots of the look-back kernels within one frame
enum : int { SLOT_CULL = 0, SLOT_SCAN = 8, SLOT_SORT1 = 12, SLOT_SORT2 = 20, SLOT_AUX = 28, SLOT_BLEND = 29, SLOT_KEYGEN = 30,
             SLOT_CACHE = 32 };
constexpr int MAX_CACHES = 16;  // two scan slots each in [SLOT_CACHE, 64)

// Frame setup; also clears ranges[0 .. n_tiles).
void launch_frame_begin(FrameDev* fd, const FrameIn* fin, CacheDev* caches, int n_caches, uint2* ranges,
                        uint32_t n_tiles, cudaStream_t s);
void launch_bump_epoch(FrameDev* fd, uint32_t spin_limit, cudaStream_t s);
void launch_wait_probe(FrameDev* fd, unsigned long long* words, cudaStream_t s);
// Anchor filtering of one model in two passes (keep masks and per-tile
// counts, then the ids): vis_dev / eyes_dev per derivation view the visible
// ids and, for exact stereo views, each one's eye mask (bit e: camera
// dview_cam[d][e] keeps it); masks [views][mask_stride] and tile_cnt
// [views][cnt_stride] are the passes' working arrays (cull_mask_words /
// cull_tiles of the model's anchors per view).  h_model: the model's device
// description as the host holds it.
// probe.caches (the frame's caches, device array, or null): the write pass
// runs the depth-rule probe of the model's views' caches as it writes each
// id, and the free flags of their lines (the probe kernel is then left out).
// Returns false (nothing launched) for a model without anchors.
struct CullProbe {
  CacheDev* caches;
};
bool launch_cull(const ModelDev* md, const ModelDev* h_model, int model, FrameDev* fd, uint32_t* const* vis_dev,
                 uint8_t* const* eyes_dev, uint32_t* masks, uint32_t* tile_cnt, uint32_t mask_stride,
                 uint32_t cnt_stride, CullProbe probe, cudaStream_t s);
uint32_t cull_tiles(uint32_t n_anchors);
uint32_t cull_mask_words(uint32_t n_anchors);
void launch_plan(FrameDev* fd, uint32_t rec_cap, cudaStream_t s);
cudaError_t prepare_derive_f32();
cudaError_t prepare_derive_tc();
cudaError_t prepare_sort();
void launch_to_bf16(const float* src, void* dst, size_t n, cudaStream_t s);
// Per-frame tables (defined in derive_common.cuh): the decoder's view set of
// each model and the projection's per-view table, written by k_tables.
struct DViewSet;
struct ProjTab;
size_t dview_set_bytes();
size_t proj_tab_bytes();
void launch_tables(const FrameDev* fd, const CacheDev* caches, uint8_t* const* eyes_dev, DViewSet* tabs,
                   ProjTab* ptab, int n_models, cudaStream_t s);
void launch_derive_tc(const ModelDev* models, int model, FrameDev* fd, uint32_t* const* vis, float4* attrs,
                      float* const* dbg_attrs, const CacheDev* caches, const DViewSet* tabs, bool fp8, int n_sm,
                      cudaStream_t s);
// FP8-E4M3 form: per-tensor power-of-two scales, the weight image, feature conversion
struct Fp8Scales {
  float sx, sw1[3], sw2[3], sh[3];
};
Fp8Scales fp8_scales(const float* feat, size_t n, const float* const W1[3], const float* const b1[3],
                     const float* const W2[3]);
constexpr size_t TC8_IMAGE_BYTES = 70016;
cudaError_t make_tc8_image(const float* const W1[3], const float* const b1[3], const float* const W2[3],
                           const float* const b2[3], const Fp8Scales& S, void* d_img, cudaStream_t s);
void launch_to_e4m3(const float* src, float inv_scale, void* dst, size_t n, cudaStream_t s);
void launch_to_e4m3_two_term(const float* src, void* hi, void* lo, size_t n, cudaStream_t s);
void pack_tc_weights(const float* const W1[3], const float* const b1[3], const float* const W2[3],
                     const float* const b2[3], std::vector<uint8_t>& img);
void launch_derive_f32(const ModelDev* models, int model, FrameDev* fd, uint32_t* const* vis, float4* attrs,
                       float* const* dbg_attrs, const CacheDev* caches, const DViewSet* tabs, int n_sm,
                       cudaStream_t s);
// The derivation as separate operators through device memory (the
// ablation's unfused decoder; float32): scratch holds
// unfused_scratch_floats(items_cap) floats, items_cap >= the decoded anchors
// of the model's views; h_model is the model's device description as the
// host holds it.
size_t unfused_scratch_floats(size_t items);
void launch_derive_unfused(const ModelDev* models, const ModelDev* h_model, int model, FrameDev* fd,
                           uint32_t* const* vis, float4* attrs, float* const* dbg_attrs, const DViewSet* tabs,
                           float* scratch, size_t items_cap, int n_sm, cudaStream_t s);
// derived attributes (3 float4 per Gaussian, frame-wide item order; cache
// hits from their lines) -> records
void launch_project(const ModelDev* models, FrameDev* fd, uint32_t* const* vis, const float4* attrs,
                    const CacheDev* caches, Records rec, const ProjTab* ptab, int n_sm, cudaStream_t s);
// Reuse-predictor training buffers (device): samples, order, parameters,
// Adam moments, gradient, per-block partials, per-epoch loss, counters
// (ctl[0] Adam steps taken, ctl[1] epoch).
struct ReuseTrain {
  const float* Z;         // [n][36]
  const float* Y;         // [n] labels 0 / 1
  const uint32_t* order;  // [epochs][n]
  float* theta;           // [2433] float32 master
  float* w;               // [2433] bfloat16-rounded copy (forward / inference)
  float* m;
  float* v;
  float* grad;
  float* part;            // [blocks][2434]
  float* loss;            // [epochs]
  uint32_t* ctl;          // [2]
};
void launch_reuse_round(const float* theta, float* w, cudaStream_t s);
int reuse_blocks(uint32_t nb);
void launch_reuse_batch(const ReuseTrain& T, uint32_t n_total, uint32_t b0, uint32_t nb, float lr, float loss_scale,
                        cudaStream_t s);
void launch_reuse_epoch_end(const ReuseTrain& T, cudaStream_t s);
// The cache kernels of a frame: probe (unless probed: the cull's write pass
// ran the depth-rule probe), collection labels, free-line scan, assignment.
void launch_cache_frame(CacheDev* caches, const CacheDev* host, int n_caches, FrameDev* fd, uint32_t* const* vis,
                        const ModelDev* models, const float* reuse_w, bool learned, const float4* attrs_fresh,
                        unsigned long long* scan_status, int n_sm, cudaStream_t s, bool probed = false);
void launch_cache_replay_counts(CacheDev* caches, int n_caches, FrameDev* fd, cudaStream_t s);
// hist: digit histograms already accumulated by the key producer (the
// histogram kernel is skipped; with drop_invalid, *n_valid_out must hold the
// kept count too), or null.
// The frame's record sort by depth (sort.cu): three 9-bit passes, and a
// fourth on bits 24-31 when fd->depth_wide; the result in (k2, v2).
void launch_depth_sort(const uint32_t* kin, uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, uint32_t* k2,
                       uint32_t* v2, const uint32_t* n_in, const uint32_t* n_valid, int slot_base, FrameDev* fd,
                       SortBufs sb, const uint32_t* hist, int n_sm, cudaStream_t s);
void launch_sort_impl(const uint32_t* kin, const uint32_t* vin, uint32_t* k0, uint32_t* v0, uint32_t* k1,
                      uint32_t* v1, const uint32_t* n_in, uint32_t* n_valid_out, int bits, int drop_invalid,
                      int slot_base, FrameDev* fd, SortBufs sb, int n_sm, cudaStream_t s, uint32_t** kout,
                      uint32_t** vout, int ipt, const uint32_t* hist = nullptr);
// Records covering more than KG_SMALL tiles get their pairs from a warp each.
constexpr uint32_t KG_SMALL = 32;
// big / n_big: indices i with cnt > big_above are appended (the large
// records of key generation), else null.  scatter_n_dev: the scatter bound
// read on the device (replaces scatter_n), else null.
void launch_scan_u32(const uint32_t* cnt, const uint32_t* order, const uint32_t* n_ptr, uint32_t* out,
                     uint32_t* total_out, unsigned long long* status, FrameDev* fd, int slot, int n_sm,
                     cudaStream_t s, uint32_t* scatter = nullptr, uint32_t scatter_n = 0, uint32_t* big = nullptr,
                     uint32_t* n_big = nullptr, uint32_t big_above = 0, const uint32_t* scatter_n_dev = nullptr);
void launch_keygen(FrameDev* fd, Records rec, const uint32_t* order, const uint32_t* offs, uint32_t* pkeys,
                   uint32_t* pvals, uint32_t cap, uint32_t* big, int n_sm, cudaStream_t s);
void launch_ranges(FrameDev* fd, const uint32_t* keys, uint2* ranges, int n_sm, cudaStream_t s);
void launch_blend(FrameDev* fd, const uint2* ranges, const uint32_t* vals, Records rec, const FrameIn* fin,
                  uint32_t total_tiles, uint32_t tile_threads, uint32_t blocks_per_sm, bool count, int n_sm,
                  cudaStream_t s);

}  // namespace gsc
