// Frame setup, anchor filtering (K1) and the per-frame plan.
#include "gsc_internal.cuh"

namespace gsc {

// ------------------------------------------------------------------ frame setup
// The cameras' constants and the derivation views (with the unified camera
// of each stereo pair, Eq. 5-6) are prepared in float64 by the library's host
// code, which has fast float64; this warp copies them into the frame plan,
// resets the per-frame counters and advances each cache's frame counter
// (lane c < n_caches, Alg. 1 tick).
__global__ void k_frame_begin(FrameDev* fd, const FrameIn* __restrict__ fin, CacheDev* __restrict__ caches,
                              int n_caches) {
  if (blockIdx.x != 0) return;
  const FrameIn& F = *fin;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t nc = F.n_cams, nd = F.n_dviews;
  if (lane < nc) {
    fd->cam[lane] = F.cam[lane];
    fd->dview_of_cam[lane] = F.dview_of_cam[lane];
  }
  if (lane < nd) {
    fd->dcam[lane] = F.dcam[lane];
    fd->dview_cam[lane][0] = F.dview_cam[lane][0];
    fd->dview_cam[lane][1] = F.dview_cam[lane][1];
    fd->dview_exact[lane] = F.dview_exact[lane];
    fd->vis_count[lane] = 0;
  }
  if (lane == 0) {
    fd->frame = fd->frame + 1;
    fd->n_cams = nc;
    fd->n_dviews = nd;
    fd->tile_w = F.tile_w;
    fd->tile_h = F.tile_h;
    fd->spin_limit = F.spin_limit;
    fd->total_tiles = F.total_tiles;
    fd->tile_bits = F.tile_bits;
    fd->cap_vis = F.cap_vis;
    fd->cap_rec = F.cap_rec;
    fd->cap_pairs = F.cap_pairs;
    fd->n_valid = 0;
    fd->n_pairs = 0;
    fd->n_pairs_used = 0;
    fd->n_big = 0;
    fd->n_derived = 0;
    fd->err = 0;
    fd->blend_work[0] = 0;
    fd->blend_work[1] = 0;
  }
  fd->ctr[lane] = 0;
  fd->ctr[32 + lane] = 0;
  {  // the two sorts' digit histograms (filled by the key producers)
    uint4* h = reinterpret_cast<uint4*>(fd->hist_depth);
    uint4* h2 = reinterpret_cast<uint4*>(fd->hist_tile);
    for (uint32_t i = lane; i < 256; i += 32) {
      h[i] = make_uint4(0, 0, 0, 0);
      h2[i] = make_uint4(0, 0, 0, 0);
    }
  }
  if ((int)lane < n_caches && caches[lane].active) {
    uint32_t* st = caches[lane].state;
    st[CS_T] += 1u;
    st[CS_MISSES] = 0;
  }
}

void launch_frame_begin(FrameDev* fd, const FrameIn* fin, CacheDev* caches, int n_caches, cudaStream_t s) {
  k_frame_begin<<<1, 32, 0, s>>>(fd, fin, caches, n_caches);
}

// New epoch for standalone uses of the look-back kernels (debug sort / scan).
__global__ void k_bump_epoch(FrameDev* fd, uint32_t spin_limit) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  fd->frame = fd->frame + 1;
  fd->spin_limit = spin_limit;
  fd->err = 0;
  fd->n_valid = 0;
  for (int i = 0; i < 64; ++i) fd->ctr[i] = 0;
}

void launch_bump_epoch(FrameDev* fd, uint32_t spin_limit, cudaStream_t s) {
  k_bump_epoch<<<1, 32, 0, s>>>(fd, spin_limit);
}

// Timeout-path probe: one thread waits, through the look-back routine, for
// a predecessor word under an epoch that no kernel ever writes.  The wait
// must give up after spin_limit polls and set ERR_TIMEOUT.
__global__ void k_wait_probe(FrameDev* fd, unsigned long long* words) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const uint32_t never = fd->frame * 64u + (uint32_t)SLOT_AUX + 7u;
  (void)lb_exclusive(words, 1, 1, never ^ 0x80000000u, fd->spin_limit, &fd->err);
}

void launch_wait_probe(FrameDev* fd, unsigned long long* words, cudaStream_t s) {
  k_wait_probe<<<1, 32, 0, s>>>(fd, words);
}

// ------------------------------------------------------------------ culling (K1)
// Anchor filtering (Sec. 3.2; Alg. 1 "anchors indexing and filtering"): for
// every derivation view of this model (for an exact stereo view: for each of
// its two cameras, the view keeping the union), frustum test with a 1.3 guard
// band and the distance LOD rule (level l >= 1 drawn iff |x - p|^2 <= (d_max 2^-l)^2,
// level 0 always; with Octree-GS level offsets the threshold is the anchor's
// own radius r_a = d_max 2^(Delta_a - l), rounded to float32 at load: the
// RADIUS instantiation).  Float32 with an explicit operation order.  Each thread
// owns CULL_IPT consecutive anchors; a block scan of per-thread counts plus a
// decoupled look-back across tiles gives an order-preserving compaction
// (ascending anchor ids), one pass over the positions.
constexpr int CULL_NT = 256;
constexpr int CULL_IPT = 8;
constexpr int CULL_TILE = CULL_NT * CULL_IPT;
constexpr int CULL_MAXD = MAXV;  // derivation views of one model (look-back words per tile)
constexpr int CULL_GROUP = 8;    // views tested together (one warp walks back per view)

template <bool RADIUS>
__global__ void __launch_bounds__(CULL_NT, 4) k_cull(const ModelDev* __restrict__ models, int model, FrameDev* fd,
                                                  uint32_t* const* __restrict__ vis, uint8_t* const* __restrict__ eyes,
                                                  unsigned long long* status) {
  __shared__ int s_d[CULL_MAXD];
  __shared__ int s_nd;
  __shared__ float s_cam[CULL_MAXD][2][20];
  __shared__ int s_ncam[CULL_MAXD];
  __shared__ float s_thr2[32];  // plain rule: (d_max 2^-l)^2 per level, +inf at level 0
  __shared__ uint32_t s_warp[CULL_NT / 32 + 1];
  __shared__ uint32_t s_total[CULL_MAXD];
  __shared__ uint32_t s_base[CULL_MAXD];
  __shared__ uint32_t s_tile;

  const ModelDev md = models[model];
  if (threadIdx.x == 0) {
    int nd = 0;
    for (uint32_t d = 0; d < fd->n_dviews; ++d) {
      if (fd->dcam[d].model != model) continue;
      if (nd < CULL_MAXD) s_d[nd++] = (int)d;
    }
    s_nd = nd;
  }
  __syncthreads();
  const int nd = s_nd;
  if (threadIdx.x < (unsigned)nd) s_ncam[threadIdx.x] = fd->dview_exact[s_d[threadIdx.x]] ? 2 : 1;
  for (int i = threadIdx.x; i < nd * 40; i += CULL_NT) {
    const int ld = i / 40, k = (i / 20) & 1, f = i % 20;
    const int d = s_d[ld];
    const bool exact = fd->dview_exact[d] != 0;
    if (k == 1 && !exact) continue;
    const CamDev& c = exact ? fd->cam[fd->dview_cam[d][k]] : fd->dcam[d];
    float v;
    if (f < 9) v = c.R[f];
    else if (f < 12) v = c.t[f - 9];
    else if (f < 15) v = c.pc[f - 12];
    else if (f == 15) v = c.znear;
    else if (f == 16) v = c.gx;
    else if (f == 17) v = c.gy;
    else v = 0.f;
    s_cam[ld][k][f] = v;
  }
  if (!RADIUS && threadIdx.x < 32) {
    const float thr = ldexpf(md.lod_dmax, -(int)threadIdx.x);
    s_thr2[threadIdx.x] = threadIdx.x == 0 ? INFINITY : __fmul_rn(thr, thr);
  }
  __syncthreads();
  if (nd == 0) return;

  const uint32_t n = md.n;
  const uint32_t ntiles = (n + CULL_TILE - 1) / CULL_TILE;
  const uint32_t epoch = fd->frame * 64u + (uint32_t)(SLOT_CULL + model);
  const uint32_t spin = fd->spin_limit;

  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&fd->ctr[SLOT_CULL + model], 1u);
    __syncthreads();
    const uint32_t t = s_tile;
    if (t >= ntiles) break;
    const uint32_t a0 = t * CULL_TILE + threadIdx.x * CULL_IPT;
    float x[CULL_IPT], y[CULL_IPT], z[CULL_IPT];
    int lv[CULL_IPT];     // plain rule: level, -1 past the end
    float rr[CULL_IPT];   // radius rule: the anchor's switching radius (+inf at level 0);
                          // past the end the position is NaN, which fails the frustum test
    static_assert(CULL_IPT == 8, "a thread loads two float4 per coordinate and 8 level bytes");
    if (a0 + CULL_IPT <= n) {  // 32-byte aligned runs (a0 is a multiple of 8; arrays are 256-byte aligned)
      const float4 x0 = __ldg(reinterpret_cast<const float4*>(md.px + a0)), x1 = __ldg(reinterpret_cast<const float4*>(md.px + a0) + 1);
      const float4 y0 = __ldg(reinterpret_cast<const float4*>(md.py + a0)), y1 = __ldg(reinterpret_cast<const float4*>(md.py + a0) + 1);
      const float4 z0 = __ldg(reinterpret_cast<const float4*>(md.pz + a0)), z1 = __ldg(reinterpret_cast<const float4*>(md.pz + a0) + 1);
      x[0] = x0.x; x[1] = x0.y; x[2] = x0.z; x[3] = x0.w; x[4] = x1.x; x[5] = x1.y; x[6] = x1.z; x[7] = x1.w;
      y[0] = y0.x; y[1] = y0.y; y[2] = y0.z; y[3] = y0.w; y[4] = y1.x; y[5] = y1.y; y[6] = y1.z; y[7] = y1.w;
      z[0] = z0.x; z[1] = z0.y; z[2] = z0.z; z[3] = z0.w; z[4] = z1.x; z[5] = z1.y; z[6] = z1.z; z[7] = z1.w;
      if (RADIUS) {
        const float4 r0 = __ldg(reinterpret_cast<const float4*>(md.lod_r + a0));
        const float4 r1 = __ldg(reinterpret_cast<const float4*>(md.lod_r + a0) + 1);
        rr[0] = r0.x; rr[1] = r0.y; rr[2] = r0.z; rr[3] = r0.w; rr[4] = r1.x; rr[5] = r1.y; rr[6] = r1.z; rr[7] = r1.w;
      } else {
        const uint2 l8 = __ldg(reinterpret_cast<const uint2*>(md.level + a0));
#pragma unroll
        for (int i = 0; i < CULL_IPT; ++i) lv[i] = (int)(((i < 4 ? l8.x : l8.y) >> (8 * (i & 3))) & 0xFFu);
      }
    } else {
#pragma unroll
      for (int i = 0; i < CULL_IPT; ++i) {
        const uint32_t a = a0 + i;
        if (a < n) {
          x[i] = __ldg(md.px + a);
          y[i] = __ldg(md.py + a);
          z[i] = __ldg(md.pz + a);
          if (RADIUS)
            rr[i] = __ldg(md.lod_r + a);
          else
            lv[i] = md.level[a];
        } else if (RADIUS) {
          x[i] = y[i] = z[i] = __int_as_float(0x7fffffff);
          rr[i] = 0.f;
        } else {
          x[i] = y[i] = z[i] = 0.f;
          lv[i] = -1;
        }
      }
    }
    for (int g0 = 0; g0 < nd; g0 += CULL_GROUP) {  // views g0 .. g0 + 7 of this model
      // mask[u]: bits 0-7 the view keeps anchor i, bits 8-15 / 16-23 its first /
      // second camera does (exact stereo views)
      uint32_t excl[CULL_GROUP], mask[CULL_GROUP];
#pragma unroll
      for (int u = 0; u < CULL_GROUP; ++u) {
        const int ld = g0 + u;
        excl[u] = 0;
        mask[u] = 0;
        if (ld >= nd) continue;
        uint32_t m = 0;
        for (int k = 0; k < s_ncam[ld]; ++k) {
          const float* c = s_cam[ld][k];
          uint32_t mk = 0;
#pragma unroll
          for (int i = 0; i < CULL_IPT; ++i) {
            if (!RADIUS && lv[i] < 0) continue;
            const float X = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c[0], x[i]), __fmul_rn(c[1], y[i])), __fmul_rn(c[2], z[i])), c[9]);
            const float Y = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c[3], x[i]), __fmul_rn(c[4], y[i])), __fmul_rn(c[5], z[i])), c[10]);
            const float Z = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c[6], x[i]), __fmul_rn(c[7], y[i])), __fmul_rn(c[8], z[i])), c[11]);
            bool v = (Z > c[15]) && (fabsf(X) <= __fmul_rn(c[16], Z)) && (fabsf(Y) <= __fmul_rn(c[17], Z));
            if (v) {
              const float dx = __fsub_rn(x[i], c[12]), dy = __fsub_rn(y[i], c[13]), dz = __fsub_rn(z[i], c[14]);
              const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
              v = d2 <= (RADIUS ? __fmul_rn(rr[i], rr[i]) : s_thr2[lv[i]]);
            }
            if (v) mk |= 1u << i;
          }
          m |= mk | (mk << (8 + 8 * k));
        }
        mask[u] = m;
        uint32_t tot;
        excl[u] = block_exclusive_scan<CULL_NT>((uint32_t)__popc(m & 0xFFu), s_warp, &tot);
        if (threadIdx.x == 0) s_total[ld] = tot;
      }
      __syncthreads();
      const int ld = g0 + (int)(threadIdx.x >> 5);
      if (ld < nd && (int)(threadIdx.x >> 5) < CULL_GROUP) {  // warp u publishes view g0 + u's count, walks back
        const bool l0 = (threadIdx.x & 31u) == 0;
        const uint32_t tot = s_total[ld];
        unsigned long long* w = status + (size_t)t * CULL_MAXD + ld;
        uint32_t pre = 0;
        if (t == 0) {
          if (l0) st_relaxed_u64(w, lb_pack(epoch, 2u, tot));
        } else {
          if (l0) st_relaxed_u64(w, lb_pack(epoch, 1u, tot));
          pre = lb_exclusive_warp(status + ld, CULL_MAXD, t, epoch, spin, &fd->err);
          if (l0) st_relaxed_u64(w, lb_pack(epoch, 2u, pre + tot));
        }
        if (l0) {
          s_base[ld] = pre;
          if (t == ntiles - 1) fd->vis_count[s_d[ld]] = pre + tot;
        }
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < CULL_GROUP; ++u) {
        const int lw = g0 + u;
        if (lw >= nd) continue;
        uint32_t* out = vis[s_d[lw]];
        uint8_t* eo = s_ncam[lw] == 2 ? eyes[s_d[lw]] : nullptr;
        uint32_t o = s_base[lw] + excl[u];
        const uint32_t mm = mask[u];
        uint32_t m = mm & 0xFFu;
        while (m) {
          const int i = __ffs(m) - 1;
          m &= m - 1;
          if (GSC_IN_BOUNDS(o, fd->cap_vis, &fd->err)) {
            if (eo) eo[o] = (uint8_t)(((mm >> (8 + i)) & 1u) | (((mm >> (16 + i)) & 1u) << 1));
            out[o] = a0 + (uint32_t)i;
          }
          ++o;
        }
      }
      __syncthreads();
    }
  }
}

void launch_cull(const ModelDev* md, int model, bool radius, FrameDev* fd, uint32_t* const* vis_dev,
                 uint8_t* const* eyes_dev, unsigned long long* status, int n_sm, cudaStream_t s) {
  if (radius)
    k_cull<true><<<n_sm * 4, CULL_NT, 0, s>>>(md, model, fd, vis_dev, eyes_dev, status);
  else
    k_cull<false><<<n_sm * 4, CULL_NT, 0, s>>>(md, model, fd, vis_dev, eyes_dev, status);
}

// ------------------------------------------------------------------ plan
__global__ void k_plan(FrameDev* fd, uint32_t rec_cap) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint32_t acc = 0;
  for (uint32_t d = 0; d < fd->n_dviews; ++d) {
    fd->item_base[d] = acc;
    acc += fd->vis_count[d];
  }
  fd->item_base[fd->n_dviews] = acc;
  fd->n_items = acc;
  fd->n_derived = acc;  // lowered by the cache policy when views reuse
  unsigned long long r = 0;
  for (uint32_t c = 0; c < fd->n_cams; ++c) {
    fd->rec_base[c] = (uint32_t)(r < 0xFFFFFFFFull ? r : 0xFFFFFFFFull);
    r += (unsigned long long)K * fd->vis_count[fd->dview_of_cam[c]];
  }
  fd->rec_base[fd->n_cams] = (uint32_t)(r < 0xFFFFFFFFull ? r : 0xFFFFFFFFull);
  fd->n_records_need = (uint32_t)(r < 0xFFFFFFFFull ? r : 0xFFFFFFFFull);
  if (r > rec_cap) {
    atomicOr(&fd->err, ERR_REC_OVERFLOW);
    fd->n_records = rec_cap;
  } else {
    fd->n_records = (uint32_t)r;
  }
}

void launch_plan(FrameDev* fd, uint32_t rec_cap, cudaStream_t s) { k_plan<<<1, 32, 0, s>>>(fd, rec_cap); }

}  // namespace gsc
