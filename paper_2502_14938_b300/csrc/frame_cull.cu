// Frame setup, anchor filtering (K1) and the per-frame plan.
#include "derive_common.cuh"

namespace gsc {

// ------------------------------------------------------------------ frame setup
// The cameras' constants and the derivation views (with the unified camera
// of each stereo pair, Eq. 5-6) are prepared in float64 by the library's host
// code, which has fast float64; block 0 copies them into the frame plan
// (word by word across its threads), resets the per-frame counters and
// histograms and advances each cache's frame counter (thread c < n_caches,
// Alg. 1 tick); every block clears its share of the tile ranges.
constexpr int FB_NT = 256;
static_assert(sizeof(CamDev) % 4 == 0, "cameras are copied as words");

__global__ void __launch_bounds__(FB_NT) k_frame_begin(FrameDev* fd, const FrameIn* __restrict__ fin,
                                                       CacheDev* __restrict__ caches, int n_caches,
                                                       uint2* __restrict__ ranges, uint32_t n_tiles) {
  // every block: its share of the tile ranges, cleared (tiles without pairs keep [0, 0))
  for (uint32_t i = blockIdx.x * FB_NT + threadIdx.x; i < n_tiles; i += gridDim.x * FB_NT) ranges[i] = make_uint2(0, 0);
  if (blockIdx.x != 0) return;
  const FrameIn& F = *fin;
  const uint32_t t = threadIdx.x;
  const uint32_t nc = F.n_cams, nd = F.n_dviews;
  {
    constexpr uint32_t CW = sizeof(CamDev) / 4;
    const uint32_t* src = reinterpret_cast<const uint32_t*>(F.cam);
    uint32_t* dst = reinterpret_cast<uint32_t*>(fd->cam);
    for (uint32_t i = t; i < nc * CW; i += FB_NT) dst[i] = src[i];
    src = reinterpret_cast<const uint32_t*>(F.dcam);
    dst = reinterpret_cast<uint32_t*>(fd->dcam);
    for (uint32_t i = t; i < nd * CW; i += FB_NT) dst[i] = src[i];
  }
  if (t < nc) fd->dview_of_cam[t] = F.dview_of_cam[t];
  if (t < nd) {
    fd->dview_cam[t][0] = F.dview_cam[t][0];
    fd->dview_cam[t][1] = F.dview_cam[t][1];
    fd->dview_exact[t] = F.dview_exact[t];
    fd->vis_count[t] = 0;
  }
  if (t == 0) {
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
    fd->depth_base = F.depth_base;
    fd->depth_wide = 0;
  }
  if (t < 64) fd->ctr[t] = 0;
  {  // the two sorts' digit histograms (filled by the key producers)
    uint4* h = reinterpret_cast<uint4*>(fd->hist_depth);
    uint4* h2 = reinterpret_cast<uint4*>(fd->hist_tile);
    static_assert(FB_NT == 256 && DEPTH_HIST_WORDS % 4 == 0, "uint4 stores");
    for (uint32_t i = t; i < DEPTH_HIST_WORDS / 4; i += FB_NT) h[i] = make_uint4(0, 0, 0, 0);
    h2[t] = make_uint4(0, 0, 0, 0);
  }
  if ((int)t < n_caches && caches[t].active) {
    uint32_t* st = caches[t].state;
    st[CS_T] += 1u;
    st[CS_MISSES] = 0;
    st[CS_HW] = st[CS_HW_NEXT];
  }
}

void launch_frame_begin(FrameDev* fd, const FrameIn* fin, CacheDev* caches, int n_caches, uint2* ranges,
                        uint32_t n_tiles, cudaStream_t s) {
  const uint32_t blocks = n_tiles > 4u * FB_NT ? (n_tiles + 4u * FB_NT - 1) / (4u * FB_NT) : 1u;
  k_frame_begin<<<blocks, FB_NT, 0, s>>>(fd, fin, caches, n_caches, ranges, n_tiles);
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

// ------------------------------------------------------------------ plan
// Item and record bases of the frame's views and cameras (one thread).
__device__ __forceinline__ void plan_thread(FrameDev* fd, uint32_t rec_cap) {
  uint32_t acc = 0;
  for (uint32_t d = 0; d < fd->n_dviews; ++d) {
    fd->item_base[d] = acc;
    acc += fd->vis_count[d];
  }
  fd->item_base[fd->n_dviews] = acc;
  fd->n_items = acc;
  atomicAdd(&fd->n_derived, acc);  // (from 0) lowered by the cache policy when views reuse, in either order
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

// ------------------------------------------------------------------ culling (K1)
// Anchor filtering (Sec. 3.2; Alg. 1 "anchors indexing and filtering"): for
// every derivation view of this model (for an exact stereo view: for each of
// its two cameras, the view keeping the union), frustum test with a 1.3 guard
// band and the distance LOD rule (level l >= 1 drawn iff |x - p|^2 <= (d_max
// 2^-l)^2, level 0 always; with Octree-GS level offsets the threshold is the
// anchor's own radius r_a = d_max 2^(Delta_a - l), rounded to float32 at
// load: the RADIUS instantiation).  Float32 with an explicit operation order.
//
// Two passes over tiles of CULL_TILE anchors (CULL_IPT consecutive anchors
// per thread), with no waits between blocks:
//   count  each thread's keep masks per view (bits 0-7 the view keeps
//          anchor i, 8-15 / 16-23 the first / second camera of an exact
//          stereo view does) to device memory, and per tile and view the
//          number kept.  A camera keeps an anchor iff both its LOD and its
//          frustum test pass; the LOD test runs first for every anchor and
//          rejects all but a few percent of a city-scale model, and each
//          warp then runs the frustum tests on its LOD survivors only, 32 at
//          a time (the same float32 operations, so the same decisions)
//   write  per tile and view the exclusive prefix of the tiles before it (a
//          block-wide sum of their counts), a block scan of the threads'
//          counts, and the kept ids in ascending order (with their eye
//          masks); the last tile sets the view's visible count.
// The order-preserving compaction is the same as a scan over all anchors.
constexpr int CULL_NT = 256;
constexpr int CULL_IPT = 8;
constexpr int CULL_TILE = CULL_NT * CULL_IPT;
constexpr int CULL_MAXD = MAXV;  // derivation views of one model

// Derivation views of this model and their cameras (shared memory), set up by every block.
struct CullViews {
  int d[CULL_MAXD];
  int ncam[CULL_MAXD];
  float cam[CULL_MAXD][2][20];
  float thr2[32];  // plain rule: (d_max 2^-l)^2 per level, +inf at level 0
  int nd;
};

template <bool RADIUS>
__device__ __forceinline__ void cull_views_setup(CullViews& V, const ModelDev& md, int model, const FrameDev* fd) {
  if (threadIdx.x == 0) {
    int nd = 0;
    for (uint32_t d = 0; d < fd->n_dviews; ++d) {
      if (fd->dcam[d].model != model) continue;
      if (nd < CULL_MAXD) V.d[nd++] = (int)d;
    }
    V.nd = nd;
  }
  __syncthreads();
  const int nd = V.nd;
  if (threadIdx.x < (unsigned)nd) V.ncam[threadIdx.x] = fd->dview_exact[V.d[threadIdx.x]] ? 2 : 1;
  for (int i = threadIdx.x; i < nd * 40; i += CULL_NT) {
    const int ld = i / 40, k = (i / 20) & 1, f = i % 20;
    const int d = V.d[ld];
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
    V.cam[ld][k][f] = v;
  }
  if (!RADIUS && threadIdx.x < 32) {
    const float thr = ldexpf(md.lod_dmax, -(int)threadIdx.x);
    V.thr2[threadIdx.x] = threadIdx.x == 0 ? INFINITY : __fmul_rn(thr, thr);
  }
  __syncthreads();
}

template <bool RADIUS>
__global__ void __launch_bounds__(CULL_NT, 4) k_cull_count(const ModelDev* __restrict__ models, int model,
                                                        const FrameDev* __restrict__ fd, uint32_t* __restrict__ masks,
                                                        uint32_t* __restrict__ tile_cnt, uint32_t mask_stride,
                                                        uint32_t cnt_stride) {
  __shared__ CullViews V;
  __shared__ uint32_t s_cnt[CULL_MAXD];
  __shared__ uint16_t s_list[CULL_NT / 32][32 * CULL_IPT];  // per warp: LOD survivors
  __shared__ uint32_t s_mask[CULL_NT];                      // per thread: keep masks being built
  const ModelDev md = models[model];
  cull_views_setup<RADIUS>(V, md, model, fd);
  const int nd = V.nd;
  if (nd == 0) return;
  if (threadIdx.x < (unsigned)nd) s_cnt[threadIdx.x] = 0;
  const uint32_t n = md.n;
  const uint32_t t = blockIdx.x;
  const uint32_t a0 = t * CULL_TILE + threadIdx.x * CULL_IPT;
  __syncthreads();  // s_cnt cleared
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint16_t* list = s_list[warp];
  for (int ld = 0; ld < nd; ++ld) {
    const int ncam = V.ncam[ld];
    // (positions are loaded per view, so that they are not live across the
    // survivor pass; a second view finds them in L1)
    float x[CULL_IPT], y[CULL_IPT], z[CULL_IPT];
    float thr[CULL_IPT];  // squared LOD distance: (d_max 2^-l)^2 from the level table, or the
                          // anchor's own radius squared; -1 past the end (never kept)
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
        const float rr[CULL_IPT] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
  #pragma unroll
        for (int i = 0; i < CULL_IPT; ++i) thr[i] = __fmul_rn(rr[i], rr[i]);
      } else {
        const uint2 l8 = __ldg(reinterpret_cast<const uint2*>(md.level + a0));
  #pragma unroll
        for (int i = 0; i < CULL_IPT; ++i) thr[i] = V.thr2[((i < 4 ? l8.x : l8.y) >> (8 * (i & 3))) & 0xFFu];
      }
    } else {
  #pragma unroll
      for (int i = 0; i < CULL_IPT; ++i) {
        const uint32_t a = a0 + i;
        x[i] = y[i] = z[i] = 0.f;
        thr[i] = -1.f;
        if (a < n) {
          x[i] = __ldg(md.px + a);
          y[i] = __ldg(md.py + a);
          z[i] = __ldg(md.pz + a);
          if (RADIUS) {
            const float r = __ldg(md.lod_r + a);
            thr[i] = __fmul_rn(r, r);
          } else {
            thr[i] = V.thr2[md.level[a]];
          }
        }
      }
    }
    // LOD of every anchor for each camera (the cheap test, which keeps a few
    // percent of the city): bit i of lod0 / lod1
    uint32_t lod0 = 0u, lod1 = 0u;
    for (int k = 0; k < ncam; ++k) {
      const float* c = V.cam[ld][k];
      const float px = c[12], py = c[13], pz = c[14];
      uint32_t lk = 0u;
#pragma unroll
      for (int i = 0; i < CULL_IPT; ++i) {
        const float dx = __fsub_rn(x[i], px), dy = __fsub_rn(y[i], py), dz = __fsub_rn(z[i], pz);
        const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
        if (d2 <= thr[i]) lk |= 1u << i;
      }
      if (k == 0) lod0 = lk; else lod1 = lk;
    }
    // the warp's LOD survivors, compacted: entry = anchor slot (lane * 8 + i)
    // | the cameras whose LOD kept it << 8
    const uint32_t cand = lod0 | lod1;
    const uint32_t nc = (uint32_t)__popc(cand);
    uint32_t inc = nc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
    uint32_t pos = inc - nc;
    for (uint32_t cm = cand; cm; cm &= cm - 1) {
      const int i = __ffs(cm) - 1;
      list[pos++] = (uint16_t)((lane << 3) | i | (((lod0 >> i) & 1u) << 8) | (((lod1 >> i) & 1u) << 9));
    }
    s_mask[threadIdx.x] = 0u;
    __syncwarp();
    // frustum tests of the survivors, 32 at a time across the warp
    for (uint32_t j = lane; j < ((total + 31u) & ~31u); j += 32u) {
      if (j < total) {
        const uint32_t e = list[j];
        const uint32_t owner = (e >> 3) & 31u, i = e & 7u;
        const uint32_t a = t * CULL_TILE + ((uint32_t)warp * 32u + owner) * CULL_IPT + i;
        const float xa = __ldg(md.px + a), ya = __ldg(md.py + a), za = __ldg(md.pz + a);
        uint32_t bits = 0;
        for (int k = 0; k < ncam; ++k) {
          if (!((e >> (8 + k)) & 1u)) continue;
          const float* c = V.cam[ld][k];
          const float X = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c[0], xa), __fmul_rn(c[1], ya)), __fmul_rn(c[2], za)), c[9]);
          const float Y = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c[3], xa), __fmul_rn(c[4], ya)), __fmul_rn(c[5], za)), c[10]);
          const float Z = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c[6], xa), __fmul_rn(c[7], ya)), __fmul_rn(c[8], za)), c[11]);
          if ((Z > c[15]) && (fabsf(X) <= __fmul_rn(c[16], Z)) && (fabsf(Y) <= __fmul_rn(c[17], Z)))
            bits |= (1u << i) | (1u << (8 + 8 * k + i));
        }
        if (bits) atomicOr(&s_mask[warp * 32 + (int)owner], bits);
      }
    }
    __syncwarp();
    const uint32_t m = s_mask[threadIdx.x];
    masks[(size_t)ld * mask_stride + (size_t)t * CULL_NT + threadIdx.x] = m;
    const uint32_t c = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(m & 0xFFu));
    if (lane == 0 && c) atomicAdd(&s_cnt[ld], c);
    __syncwarp();  // s_mask and the list are reused by the next view
  }
  __syncthreads();
  if (threadIdx.x < (unsigned)nd) tile_cnt[(size_t)threadIdx.x * cnt_stride + t] = s_cnt[threadIdx.x];
}

__global__ void __launch_bounds__(CULL_NT, 4) k_cull_write(const ModelDev* __restrict__ models, int model,
                                                        FrameDev* __restrict__ fd, uint32_t* const* __restrict__ vis,
                                                        uint8_t* const* __restrict__ eyes,
                                                        const uint32_t* __restrict__ masks,
                                                        const uint32_t* __restrict__ tile_cnt, uint32_t mask_stride,
                                                        uint32_t cnt_stride, CullProbe probe_cfg) {
  __shared__ int s_d[CULL_MAXD];
  __shared__ int s_exact[CULL_MAXD];
  __shared__ int s_nd;
  __shared__ uint32_t s_warp[CULL_NT / 32 + 1];
  __shared__ uint32_t s_red[CULL_NT / 32];
  const ModelDev& md = models[model];
  if (threadIdx.x == 0) {
    int nd = 0;
    for (uint32_t d = 0; d < fd->n_dviews; ++d) {
      if (fd->dcam[d].model != model) continue;
      if (nd < CULL_MAXD) {
        s_exact[nd] = fd->dview_exact[d];
        s_d[nd++] = (int)d;
      }
    }
    s_nd = nd;
  }
  __syncthreads();
  const int nd = s_nd;
  const uint32_t t = blockIdx.x;
  const uint32_t ntiles = (md.n + CULL_TILE - 1) / CULL_TILE;
  const uint32_t a0 = t * CULL_TILE + threadIdx.x * CULL_IPT;
  for (int ld = 0; ld < nd; ++ld) {
    const int d = s_d[ld];
    // the view's cache, probed by the depth rule as each id is written
    const bool probe = probe_cfg.caches && d < MAX_CACHES && probe_cfg.caches[d].active;
    CacheDev cd{};
    uint32_t ct = 0, cdepth = 0, cD = 0, chw = 0;
    if (probe) {
      cd = probe_cfg.caches[d];
      ct = cd.state[CS_T];
      cdepth = cd.state[CS_DEPTH];
      cD = cd.state[CS_DMAX];
      chw = cd.state[CS_HW];
    }
    // prefix of the tiles before this one: a block-wide sum of their counts
    const uint32_t* tc = tile_cnt + (size_t)ld * cnt_stride;
    uint32_t p = 0;
    for (uint32_t u = threadIdx.x; u < t; u += CULL_NT) p += tc[u];
    p = __reduce_add_sync(0xffffffffu, p);
    if ((threadIdx.x & 31u) == 0) s_red[threadIdx.x >> 5] = p;
    const uint32_t m = masks[(size_t)ld * mask_stride + (size_t)t * CULL_NT + threadIdx.x];
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan<CULL_NT>((uint32_t)__popc(m & 0xFFu), s_warp, &tot);  // syncs
    uint32_t pre = 0;
#pragma unroll
    for (int w = 0; w < CULL_NT / 32; ++w) pre += s_red[w];
    uint32_t* out = vis[d];
    uint8_t* eo = s_exact[ld] ? eyes[d] : nullptr;
    uint32_t o = pre + ex;
    uint32_t mm = m & 0xFFu;
    while (mm) {
      const int i = __ffs(mm) - 1;
      mm &= mm - 1;
      if (GSC_IN_BOUNDS(o, fd->cap_vis, &fd->err)) {
        const uint32_t a = a0 + (uint32_t)i;
        if (eo) eo[o] = (uint8_t)(((m >> (8 + i)) & 1u) | (((m >> (16 + i)) & 1u) << 1));
        out[o] = a;
        if (probe) cache_probe_depth(cd, a, o, ct, cdepth, cD, chw, fd->cap_vis, &fd->err);
      }
      ++o;
    }
    if (probe)  // free flags of the lines below the high-water mark, spread over the blocks
      for (uint32_t l = t * CULL_NT + threadIdx.x; l < chw; l += gridDim.x * CULL_NT) cd.flags[l] = cache_line_free(cd, l, ct, cD);
    if (t == ntiles - 1 && threadIdx.x == 0) {
      fd->vis_count[d] = pre + tot;
      if (probe) cd.state[CS_SCAN_N] = chw + pre + tot;
    }
    __syncthreads();  // s_red is reused by the next view
  }
}

bool launch_cull(const ModelDev* md, const ModelDev* h_model, int model, FrameDev* fd, uint32_t* const* vis_dev,
                 uint8_t* const* eyes_dev, uint32_t* masks, uint32_t* tile_cnt, uint32_t mask_stride,
                 uint32_t cnt_stride, CullProbe probe, cudaStream_t s) {
  const uint32_t ntiles = (h_model->n + CULL_TILE - 1) / CULL_TILE;
  if (ntiles == 0) return false;
  if (h_model->lod_r)
    k_cull_count<true><<<ntiles, CULL_NT, 0, s>>>(md, model, fd, masks, tile_cnt, mask_stride, cnt_stride);
  else
    k_cull_count<false><<<ntiles, CULL_NT, 0, s>>>(md, model, fd, masks, tile_cnt, mask_stride, cnt_stride);
  k_cull_write<<<ntiles, CULL_NT, 0, s>>>(md, model, fd, vis_dev, eyes_dev, masks, tile_cnt, mask_stride, cnt_stride,
                                          probe);
  return true;
}

uint32_t cull_tiles(uint32_t n_anchors) { return (n_anchors + CULL_TILE - 1) / CULL_TILE; }
uint32_t cull_mask_words(uint32_t n_anchors) { return cull_tiles(n_anchors) * CULL_NT; }

__global__ void k_plan(FrameDev* fd, uint32_t rec_cap) {
  if (threadIdx.x == 0 && blockIdx.x == 0) plan_thread(fd, rec_cap);
}

void launch_plan(FrameDev* fd, uint32_t rec_cap, cudaStream_t s) { k_plan<<<1, 32, 0, s>>>(fd, rec_cap); }

}  // namespace gsc
