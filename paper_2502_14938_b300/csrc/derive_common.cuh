// Pieces shared by the derivation kernels (float32 CUDA-core and tcgen05
// tensor-core): the per-block list of derivation views, the activation
// epilogue of Eq. 3 and the EWA projection + exact tile count (Eq. 1-2,
// Sec. 6) that turns one derived Gaussian into one record per camera.
#pragma once
#include <cuda_fp16.h>

#include "gsc_internal.cuh"

namespace gsc {

struct ProjCam {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  float znear, gx, gy;
  float pc[3], pc_lo[3], dt[3];
  int W, H;
  uint32_t rec_base;
  uint32_t cam;
};

// Derivation views of one model, staged in shared memory by one thread.
struct DViewSet {
  int nd;
  int d[MAXV];
  uint32_t base[MAXV + 1];  // prefix of visible counts over the listed views
  uint32_t gbase[MAXV];     // frame-wide item index of each listed view's first anchor
  const uint32_t* miss[MAXV];  // cached views: visible indices to decode (else null: all)
  const uint32_t* vstat[MAXV]; // cached views: line status per visible index
  uint2* lattr[MAXV];          // cached views: float16 line attributes
  float pc[MAXV][6];        // double-float centre of each derivation camera
};

// Per-frame tables in device memory, written once by k_tables so that the
// derivation and projection kernels stage them with one block-wide copy
// instead of each block walking the frame description serially.
struct ProjTab {              // every derivation view, for the projection
  uint32_t ibase[MAXV + 1];   // frame-wide item index of each view's first anchor; [n] = n_items
  int model[MAXV];
  const uint32_t* vstat[MAXV];
  const uint2* lattr[MAXV];
  const uint8_t* eyes[MAXV];  // exact stereo views: eye mask per visible anchor (else null)
  ProjCam cam[MAXV][2];
};

// Block-wide copy of a table (sizes are multiples of 4 bytes).
template <typename T>
__device__ __forceinline__ void stage_table(T& dst, const T* __restrict__ src) {
  static_assert(sizeof(T) % 4 == 0, "table size");
  const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d = reinterpret_cast<uint32_t*>(&dst);
  for (uint32_t i = threadIdx.x; i < sizeof(T) / 4; i += blockDim.x) d[i] = s[i];
}

__device__ __forceinline__ void fill_projcam(ProjCam& pc, const FrameDev* fd, int ci) {
  pc.cam = ci < 0 ? 0xFFFFFFFFu : (uint32_t)ci;
  if (ci < 0) return;
  const CamDev& c = fd->cam[ci];
  for (int i = 0; i < 9; ++i) pc.R[i] = c.R[i];
  for (int i = 0; i < 3; ++i) {
    pc.t[i] = c.t[i];
    pc.pc[i] = c.pc[i];
    pc.pc_lo[i] = c.pc_lo[i];
    pc.dt[i] = c.dt[i];
  }
  pc.fx = c.fx; pc.fy = c.fy; pc.cx = c.cx; pc.cy = c.cy;
  pc.znear = c.znear; pc.gx = c.gx; pc.gy = c.gy;
  pc.W = c.W; pc.H = c.H;
  pc.rec_base = fd->rec_base[ci];
}

// Work of the decoder: every visible anchor of the model's views, or for a
// view with a cache only its misses.  (One thread; k_tables builds the same
// sets for all models in parallel.)
__device__ __forceinline__ void build_dview_set(DViewSet& S, const FrameDev* fd, int model,
                                                const CacheDev* caches) {
  int nd = 0;
  uint32_t acc = 0;
  for (uint32_t d = 0; d < fd->n_dviews; ++d) {
    if (fd->dcam[d].model != model) continue;
    S.d[nd] = (int)d;
    S.base[nd] = acc;
    S.gbase[nd] = fd->item_base[d];
    const bool cached = caches && d < (uint32_t)MAX_CACHES && caches[d].active;
    S.miss[nd] = cached ? caches[d].miss : nullptr;
    S.vstat[nd] = cached ? caches[d].vstat : nullptr;
    S.lattr[nd] = cached ? caches[d].slot_attr : nullptr;
    acc += cached ? caches[d].state[CS_MISSES] : fd->vis_count[d];
    for (int u = 0; u < 3; ++u) {
      S.pc[nd][u] = fd->dcam[d].pc[u];
      S.pc[nd][3 + u] = fd->dcam[d].pc_lo[u];
    }
    ++nd;
  }
  S.base[nd] = acc;
  S.nd = nd;
}

// The decoder's view set of `model`: staged from the frame table when there
// is one, else built by thread 0.  Ends with a block barrier.
__device__ __forceinline__ void load_dview_set(DViewSet& S, const DViewSet* __restrict__ tabs, const FrameDev* fd,
                                               int model, const CacheDev* caches) {
  if (tabs)
    stage_table(S, tabs + model);
  else if (threadIdx.x == 0)
    build_dview_set(S, fd, model, caches);
  __syncthreads();
}

// The frame's tables, by one warp (lane = its lane) once the visible sets,
// the plan and the cache decisions are final: lane d fills derivation view
// d's entries of the projection table and of its model's decoder view set
// (at its rank among the model's views); lane m closes model m's set.
__device__ __forceinline__ void frame_tables_warp(const FrameDev* __restrict__ fd, const CacheDev* __restrict__ caches,
                                                  uint8_t* const* __restrict__ eyes, DViewSet* __restrict__ tabs,
                                                  ProjTab* __restrict__ ptab, int n_models, int lane) {
  const int nd = (int)fd->n_dviews;
  auto work = [&](int d) -> uint32_t {
    const bool cached = caches && d < MAX_CACHES && caches[d].active;
    return cached ? caches[d].state[CS_MISSES] : fd->vis_count[d];
  };
  if (lane < nd) {
    const int d = lane, m = fd->dcam[d].model;
    const bool cached = caches && d < MAX_CACHES && caches[d].active;
    const uint32_t ib = fd->item_base[d];
    ptab->ibase[d] = ib;
    ptab->model[d] = m;
    ptab->vstat[d] = cached ? caches[d].vstat : nullptr;
    ptab->lattr[d] = cached ? caches[d].slot_attr : nullptr;
    ptab->eyes[d] = fd->dview_exact[d] ? eyes[d] : nullptr;
    int r = 0;
    uint32_t acc = 0;
    for (int e = 0; e < d; ++e)
      if (fd->dcam[e].model == m) {
        ++r;
        acc += work(e);
      }
    DViewSet& S = tabs[m];
    S.d[r] = d;
    S.base[r] = acc;
    S.gbase[r] = ib;
    S.miss[r] = cached ? caches[d].miss : nullptr;
    S.vstat[r] = cached ? caches[d].vstat : nullptr;
    S.lattr[r] = cached ? caches[d].slot_attr : nullptr;
    for (int u = 0; u < 3; ++u) {
      S.pc[r][u] = fd->dcam[d].pc[u];
      S.pc[r][3 + u] = fd->dcam[d].pc_lo[u];
    }
    for (int e = 0; e < 2; ++e) fill_projcam(ptab->cam[d][e], fd, fd->dview_cam[d][e]);
  }
  if (lane == 0) ptab->ibase[nd] = fd->n_items;
  if (lane < n_models) {
    int c = 0;
    uint32_t tot = 0;
    for (int d = 0; d < nd; ++d)
      if (fd->dcam[d].model == lane) {
        ++c;
        tot += work(d);
      }
    tabs[lane].nd = c;
    tabs[lane].base[c] = tot;
  }
}

// EWA projection of one Gaussian + opacity-aware exact tile count.
// Decisions use the pinned depth: mu32 = x_a + o (float32 adds) and
// tz = ((R6 mu_x + R7 mu_y) + R8 mu_z) + t2 without contraction (the order
// the oracle uses for its ordering depth).  The geometry uses camera-relative
// coordinates rel = ((x_a - c_hi) - c_lo) + o, which avoid the cancellation of
// R x + t at city scale.
// The pinned ordering depth of a Gaussian at mu.
__device__ __forceinline__ float pinned_tz(const ProjCam& c, const float mu[3]) {
  return __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c.R[6], mu[0]), __fmul_rn(c.R[7], mu[1])), __fmul_rn(c.R[8], mu[2])),
                   c.t[2]);
}
// The record's first test (kept, in front of the near plane, opacity at
// least 1/255): records that fail it are only their invalid key.
__device__ __forceinline__ bool record_may_draw(const ProjCam& c, const float mu[3], float alpha, bool kept) {
  return kept && (pinned_tz(c, mu) > c.znear) && (alpha >= (1.0f / 255.0f));
}

__device__ __forceinline__ uint32_t project_write(const ProjCam& c, Records rec, uint32_t r, const float mu[3],
                                              const float rel[3], float alpha, bool kept, const float col[3],
                                              const float s[3], const float q[4], int TW, int TH) {
  const float tz = pinned_tz(c, mu);
  float4 geo = make_float4(0.f, 0.f, 0.f, 0.f), cop = make_float4(0.f, 0.f, 0.f, tz);
  uint32_t flag = c.cam;
  uint32_t cnt = 0;
  float4 colv = make_float4(col[0], col[1], col[2], 0.f);
  const bool valid = record_may_draw(c, mu, alpha, kept);
  if (valid) {
    // camera coordinates R mu + t as R (mu - pc) + (t + R pc): the large
    // parts cancel exactly in the camera-relative position
    const float tx = c.R[0] * rel[0] + c.R[1] * rel[1] + c.R[2] * rel[2] + c.dt[0];
    const float ty = c.R[3] * rel[0] + c.R[4] * rel[1] + c.R[5] * rel[2] + c.dt[1];
    const float tza = c.R[6] * rel[0] + c.R[7] * rel[1] + c.R[8] * rel[2] + c.dt[2];
    const float iz = 1.0f / tza;
    const float txc = fminf(fmaxf(tx * iz, -c.gx), c.gx) * tza;
    const float tyc = fminf(fmaxf(ty * iz, -c.gy), c.gy) * tza;
    const float j00 = c.fx * iz, j02 = -c.fx * txc * iz * iz;
    const float j11 = c.fy * iz, j12 = -c.fy * tyc * iz * iz;
    float T0[3], T1[3];  // T = J W (2x3)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      T0[k] = j00 * c.R[k] + j02 * c.R[6 + k];
      T1[k] = j11 * c.R[3 + k] + j12 * c.R[6 + k];
    }
    const float w = q[0], x = q[1], y = q[2], z = q[3];
    const float Rq[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                         2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                         2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
    float U0[3], U1[3];  // U = T R(q) diag(s); Sigma' = U U^T + 0.3 I
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float m0 = Rq[k] * s[k], m1 = Rq[3 + k] * s[k], m2 = Rq[6 + k] * s[k];
      U0[k] = T0[0] * m0 + T0[1] * m1 + T0[2] * m2;
      U1[k] = T1[0] * m0 + T1[1] * m1 + T1[2] * m2;
    }
    const float a = U0[0] * U0[0] + U0[1] * U0[1] + U0[2] * U0[2] + 0.3f;
    const float b = U0[0] * U1[0] + U0[1] * U1[1] + U0[2] * U1[2];
    const float cc = U1[0] * U1[0] + U1[1] * U1[1] + U1[2] * U1[2] + 0.3f;
    const float det = a * cc - b * b;
    if (det > 0.f) {
      const float id = 1.0f / det;
      const float A = cc * id, B = -b * id, C = a * id;
      const float mx = c.fx * tx * iz + c.cx, my = c.fy * ty * iz + c.cy;
      const float tau = 2.0f * logf(255.0f * alpha);
      const float tauc = tau * (1.0f + 0.0009765625f) + 0.0009765625f;
      geo = make_float4(mx, my, A, B);
      cop = make_float4(C, alpha, tauc, tz);
      cnt = cover_count_f32(mx, my, A, B, C, tauc, c.W, c.H, TW, TH);
      flag |= REC_VALID_BIT;
    }
  }
  // a record that covers no tile is only its invalid key: nothing reads the rest
  const uint32_t key = cnt > 0 ? __float_as_uint(tz) : INVALID_KEY;
  rec.key[r] = key;
  if (cnt > 0) {
    colv.w = __uint_as_float(flag);
    rec.geo[r] = geo;
    rec.cop[r] = cop;
    rec.col[r] = colv;
    rec.cnt[r] = cnt;
    // what every warp of every tile the record reaches would otherwise
    // recompute: the opacity in the exp2 domain and the half extents of the
    // opacity-aware box (q <= tau reaches x_mean +- sqrt(tau C / det) and
    // y_mean +- sqrt(tau A / det), det the conic's determinant)
    const float A = geo.z, B = geo.w, C = cop.x, tau = cop.z;
    const float idet = 1.f / (A * C - B * B);
    rec.aux[r] = make_float4(C, __log2f(alpha), sqrtf(tau * C * idet), sqrtf(tau * A * idet));
  }
  return key;
}

// Activations of Eq. 3 for Gaussian j of one anchor from its 11 head
// outputs z = [op_j, col_3j..3j+2, cov_7j..7j+6]:
//   alpha = tanh(z_op) (the Gaussian is kept iff alpha > 0), c = sigmoid(z_col),
//   s = s_a sigmoid(z_cov[0..2]) (the per-anchor scale broadcast to the
//   Gaussian), q = z_cov[3..6] / |.| (identity below 1e-12).
// Stored as 3 float4 at attrs[3 idx ..]: (alpha, c), (s, q_w), (q_x, q_y, q_z, 0),
// and as 12 float16 (round to nearest even) at line[0..2] when given.
// dbg (optional): the 11 attributes at dbg[11 (i K + j)].
// FAST (the tensor-core forms): sigmoid(x) = 1 / (1 + 2^(-x log2 e)) and
// tanh(x) = 2 sigmoid(2x) - 1 (odd series near 0) from the exp2 and reciprocal approximations of
// the special-function unit (__expf, __fdividef; relative errors ~1e-6, far
// inside those forms' rounding of inputs, weights and hidden layer) instead
// of the correctly rounded library sequences: the epilogue of a tile has
// only 8 warps per CTA, so its dependent instruction chains set its time.
__device__ __forceinline__ uint32_t pack_half2(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ float sigmoid_fast(float x) {
  return __fdividef(1.0f, 1.0f + __expf(-fminf(fmaxf(x, -80.f), 80.f)));
}
// tanh(x); near 0 its odd series x - x^3/3 (error below 2^-34 x for
// |x| < 2^-6), so that the sign, which carries the Gaussian's mask, is x's
__device__ __forceinline__ float tanh_fast(float x) {
  return fabsf(x) < 0.015625f ? x - x * x * x * (1.0f / 3.0f) : 2.0f * sigmoid_fast(2.0f * x) - 1.0f;
}

template <bool FAST = false>
__device__ __forceinline__ void gaussian_activate_store(const float z[11], int j, uint32_t i, float sa, float4* attrs,
                                                        size_t idx, float* dbg, uint2* line = nullptr) {
  const float alpha = FAST ? tanh_fast(z[0]) : tanhf(z[0]);
  float col[3], s[3], q[4];
#pragma unroll
  for (int u = 0; u < 3; ++u) col[u] = FAST ? sigmoid_fast(z[1 + u]) : 1.0f / (1.0f + expf(-z[1 + u]));
#pragma unroll
  for (int u = 0; u < 3; ++u) s[u] = sa * (FAST ? sigmoid_fast(z[4 + u]) : 1.0f / (1.0f + expf(-z[4 + u])));
  const float qn2 = z[7] * z[7] + z[8] * z[8] + z[9] * z[9] + z[10] * z[10];
  if (qn2 < 1e-24f) {
    q[0] = 1.f; q[1] = q[2] = q[3] = 0.f;
  } else {
    const float iq = FAST ? rsqrtf(qn2) : 1.0f / sqrtf(qn2);
#pragma unroll
    for (int u = 0; u < 4; ++u) q[u] = z[7 + u] * iq;
  }
  // alpha carries the mask: tanh(z) > 0 exactly when z > 0
  const float am = z[0] > 0.f ? alpha : -1.f;
  attrs[3 * idx + 0] = make_float4(am, col[0], col[1], col[2]);
  attrs[3 * idx + 1] = make_float4(s[0], s[1], s[2], q[0]);
  attrs[3 * idx + 2] = make_float4(q[1], q[2], q[3], 0.f);
  if (line) {
    line[0] = make_uint2(pack_half2(am, col[0]), pack_half2(col[1], col[2]));
    line[1] = make_uint2(pack_half2(s[0], s[1]), pack_half2(s[2], q[0]));
    line[2] = make_uint2(pack_half2(q[1], q[2]), pack_half2(q[3], 0.f));
  }
  if (dbg) {
    float* o = dbg + ((size_t)i * K + j) * 11;
    o[0] = alpha;
    o[1] = col[0]; o[2] = col[1]; o[3] = col[2];
    o[4] = s[0]; o[5] = s[1]; o[6] = s[2];
    o[7] = q[0]; o[8] = q[1]; o[9] = q[2]; o[10] = q[3];
  }
}

}  // namespace gsc
