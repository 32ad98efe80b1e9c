// Splatting back half: pair offsets (K6), key generation (K7), tile ranges
// (K9) and front-to-back alpha blending (K10).  Sec. 3.1 (tile
// rasterisation), Sec. 6 (opacity-aware extent, exact tile coverage).
#include "gsc_internal.cuh"

namespace gsc {

// ------------------------------------------------------------------ scan (K6)
// Exclusive prefix sum of cnt[order[i]] (or cnt[i] without order) for
// i < *n_ptr, one pass with a decoupled look-back; *total_out = the sum.
// With scatter: for i < scatter_n (or *scatter_n_dev) with cnt[i] = 1,
// scatter[out[i]] = i (the positions of the set flags, in ascending order).  With big: every i whose
// count exceeds big_above is appended to big (order unspecified).
constexpr int SCAN_NT = 256;
constexpr int SCAN_IPT = 4;  // 1024-element tiles: a frame's ~0.5M counts spread over every SM
constexpr int SCAN_TILE = SCAN_NT * SCAN_IPT;

__global__ void __launch_bounds__(SCAN_NT) k_scan(const uint32_t* __restrict__ cnt, const uint32_t* __restrict__ order,
                                                  const uint32_t* __restrict__ n_ptr, uint32_t* __restrict__ out,
                                                  uint32_t* total_out, unsigned long long* status, FrameDev* fd,
                                                  int slot, uint32_t* __restrict__ scatter, uint32_t scatter_n,
                                                  uint32_t* __restrict__ big, uint32_t* __restrict__ n_big,
                                                  uint32_t big_above, const uint32_t* __restrict__ scatter_n_dev) {
  __shared__ uint32_t s_warp[SCAN_NT / 32 + 1];
  __shared__ uint32_t s_base;
  __shared__ uint32_t s_tile;
  const uint32_t n = *n_ptr;
  if (scatter_n_dev) scatter_n = *scatter_n_dev;
  const uint32_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  const uint32_t epoch = fd->frame * 64u + (uint32_t)slot;
  const uint32_t spin = fd->spin_limit;
  if (n == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *total_out = 0;
    return;
  }
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&fd->ctr[slot], 1u);
    __syncthreads();
    const uint32_t t = s_tile;
    if (t >= ntiles) break;
    const uint32_t i0 = t * SCAN_TILE + threadIdx.x * SCAN_IPT;
    uint32_t v[SCAN_IPT];
    uint32_t sum = 0;
#pragma unroll
    for (int u = 0; u < SCAN_IPT; ++u) {
      const uint32_t i = i0 + u;
      uint32_t c = 0;
      if (i < n) c = order ? cnt[order[i]] : cnt[i];
      v[u] = c;
      sum += c;
    }
    uint32_t tot;
    uint32_t ex = block_exclusive_scan<SCAN_NT>(sum, s_warp, &tot);
    if (threadIdx.x < 32) {  // warp 0 publishes the tile and walks back
      const bool l0 = threadIdx.x == 0;
      unsigned long long* w = status + t;
      uint32_t pre = 0;
      if (t == 0) {
        if (l0) st_relaxed_u64(w, lb_pack(epoch, 2u, tot));
      } else {
        if (l0) st_relaxed_u64(w, lb_pack(epoch, 1u, tot));
        pre = lb_exclusive_warp(status, 1, t, epoch, spin, &fd->err);
        if (l0) st_relaxed_u64(w, lb_pack(epoch, 2u, pre + tot));
      }
      if (l0) {
        s_base = pre;
        if (t == ntiles - 1) *total_out = pre + tot;
      }
    }
    __syncthreads();
    uint32_t run = s_base + ex;
#pragma unroll
    for (int u = 0; u < SCAN_IPT; ++u) {
      const uint32_t i = i0 + u;
      if (i < n) {
        out[i] = run;
        if (scatter && i < scatter_n && v[u] && GSC_IN_BOUNDS(run, scatter_n, &fd->err)) scatter[run] = i;
        if (big && v[u] > big_above) {
          const uint32_t b = atomicAdd(n_big, 1u);
          if (GSC_IN_BOUNDS(b, fd->cap_rec, &fd->err)) big[b] = i;
        }
      }
      run += v[u];
    }
    __syncthreads();
  }
}

void launch_scan_u32(const uint32_t* cnt, const uint32_t* order, const uint32_t* n_ptr, uint32_t* out,
                     uint32_t* total_out, unsigned long long* status, FrameDev* fd, int slot, int n_sm,
                     cudaStream_t s, uint32_t* scatter, uint32_t scatter_n, uint32_t* big, uint32_t* n_big,
                     uint32_t big_above, const uint32_t* scatter_n_dev) {
  k_scan<<<n_sm * 4, SCAN_NT, 0, s>>>(cnt, order, n_ptr, out, total_out, status, fd, slot, scatter, scatter_n, big,
                                      n_big, big_above, scatter_n_dev);
}

// ------------------------------------------------------------------ key generation (K7)
// For the i-th record in depth order, emit (tile_base(camera) + tile, record)
// at offs[i] .. offs[i] + cnt - 1, tiles in row-major order of the exact
// coverage.  Pairs beyond the capacity are not written and flag an overflow.
// Records covering more than KG_SMALL tiles (near-camera Gaussians, up to
// thousands of tiles, clustered at the front of the depth order) were listed
// by the offset scan; each warp first takes such records one at a time: lane
// l computes the range of tile row ty0 + l (32 rows at once), a warp scan
// gives each row's offset, and the lanes write the tiles of each row.  Then
// every thread emits the small records of a grid-stride range itself.  The
// float32 row ranges are the ones the count pass used, so the pairs and their
// order are the same either way.  Then the warps take the small records in
// chunks of 32 (one per lane) from a counter, so warps that spent long on
// large records take fewer.  Each block also accumulates the digit
// histograms of the written tile keys for the tile sort (a row of a large
// record shares its upper digits: one atomic per distinct digit of a warp).
__device__ __forceinline__ void tile_hist_add(uint32_t (*s_h)[256], int npass, uint32_t key) {
  for (int p = 0; p < npass; ++p) atomicAdd(&s_h[p][(key >> (8 * p)) & 0xFFu], 1u);
}

__global__ void __launch_bounds__(256) k_keygen(FrameDev* __restrict__ fd, Records rec, const uint32_t* __restrict__ order,
                                                const uint32_t* __restrict__ offs, uint32_t* __restrict__ pkeys,
                                                uint32_t* __restrict__ pvals, uint32_t cap,
                                                const uint32_t* __restrict__ big) {
  __shared__ uint32_t s_h[4][256];
  for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) (&s_h[0][0])[i] = 0;
  const uint32_t n = fd->n_valid;
  const int npass = (int)((fd->tile_bits + 7u) / 8u);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const uint32_t np = fd->n_pairs;
    fd->n_pairs_used = np < cap ? np : cap;
    if (np > cap) atomicOr(&fd->err, ERR_PAIR_OVERFLOW);
  }
  __syncthreads();
  const int TW = (int)fd->tile_w, TH = (int)fd->tile_h;
  // large records: one warp each
  const uint32_t nb = fd->n_big;
  const uint32_t lane = threadIdx.x & 31u;
  for (;;) {
    uint32_t e = 0;
    if (lane == 0) e = atomicAdd(&fd->ctr[SLOT_AUX], 1u);
    e = __shfl_sync(0xffffffffu, e, 0);
    if (e >= nb) break;
    const uint32_t i = big[e];
    const uint32_t r = order[i];
    uint32_t o = offs[i];
    const float4 g = rec.geo[r];
    const float4 cp = rec.cop[r];
    const CamDev& cd = fd->cam[__float_as_uint(rec.col[r].w) & 0xFFFFu];
    const uint32_t tb = cd.tile_base;
    Cover cv;
    if (!cover_setup(cv, g.x, g.y, g.z, g.w, cp.x, cp.z, cd.W, cd.H, TW, TH)) continue;
    for (int c0 = cv.ty0; c0 <= cv.ty1; c0 += 32) {
      const int ty = c0 + (int)lane;
      int tx0 = 1, tx1 = 0;
      if (ty <= cv.ty1) cover_row(cv, ty, TH, tx0, tx1);
      const uint32_t len = tx1 >= tx0 ? (uint32_t)(tx1 - tx0 + 1) : 0u;
      uint32_t incl = len;
#pragma unroll
      for (int s = 1; s < 32; s <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, s);
        if (lane >= (uint32_t)s) incl += y;
      }
      const uint32_t excl = incl - len;
      const uint32_t chunk = __shfl_sync(0xffffffffu, incl, 31);
      const int rows = min(32, cv.ty1 - c0 + 1);
      for (int rr = 0; rr < rows; ++rr) {
        const uint32_t l = __shfl_sync(0xffffffffu, len, rr);
        const uint32_t ex = __shfl_sync(0xffffffffu, excl, rr);
        const int x0 = __shfl_sync(0xffffffffu, tx0, rr);
        const uint32_t kb = tb + (uint32_t)((c0 + rr) * cv.ntx + x0);
        for (uint32_t u0 = 0; u0 < l; u0 += 32u) {  // warp-uniform bounds: every lane takes part
          const uint32_t u = u0 + lane, oi = o + ex + u, key = kb + u;
          const bool w = u < l && oi < cap;
          if (w) {
            pkeys[oi] = key;
            pvals[oi] = r;
            atomicAdd(&s_h[0][key & 0xFFu], 1u);
          }
          for (int p = 1; p < npass; ++p) {
            const uint32_t d = (key >> (8 * p)) & 0xFFu;
            const unsigned peers = __match_any_sync(0xffffffffu, w ? d : 0x100u);
            if (w && (peers & ((1u << lane) - 1u)) == 0) atomicAdd(&s_h[p][d], (uint32_t)__popc(peers));
          }
        }
      }
      o += chunk;
    }
  }
  // small records: one thread each, chunks of 32 per warp from a counter
  for (;;) {
    uint32_t c = 0;
    if (lane == 0) c = atomicAdd(&fd->ctr[SLOT_KEYGEN], 1u);
    c = __shfl_sync(0xffffffffu, c, 0);
    if (c * 32u >= n) break;
    const uint32_t i = c * 32u + lane;
    if (i >= n) continue;
    const uint32_t r = order[i];
    if (rec.cnt[r] > KG_SMALL) continue;
    uint32_t o = offs[i];
    const float4 g = rec.geo[r];
    const float4 cp = rec.cop[r];
    const CamDev& cd = fd->cam[__float_as_uint(rec.col[r].w) & 0xFFFFu];
    const uint32_t tb = cd.tile_base;
    cover_tiles_f32(g.x, g.y, g.z, g.w, cp.x, cp.z, cd.W, cd.H, TW, TH, [&](int tile) {
      if (o < cap) {
        pkeys[o] = tb + (uint32_t)tile;
        pvals[o] = r;
        tile_hist_add(s_h, npass, tb + (uint32_t)tile);
      }
      ++o;
    });
  }
  __syncthreads();
  for (int i = threadIdx.x; i < npass * 256; i += blockDim.x) {
    const uint32_t c = (&s_h[0][0])[i];
    if (c) atomicAdd(&fd->hist_tile[i], c);
  }
}

void launch_keygen(FrameDev* fd, Records rec, const uint32_t* order, const uint32_t* offs, uint32_t* pkeys,
                   uint32_t* pvals, uint32_t cap, uint32_t* big, int n_sm, cudaStream_t s) {
  k_keygen<<<n_sm * 8, 256, 0, s>>>(fd, rec, order, offs, pkeys, pvals, cap, big);
}

// ------------------------------------------------------------------ tile ranges (K9)
__global__ void k_ranges(const FrameDev* __restrict__ fd, const uint32_t* __restrict__ keys, uint2* __restrict__ ranges) {
  const uint32_t n = fd->n_pairs_used;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t k = keys[i];
    if (!GSC_IN_BOUNDS(k, fd->total_tiles, const_cast<uint32_t*>(&fd->err))) continue;
    if (i == 0 || keys[i - 1] != k) ranges[k].x = i;
    if (i == n - 1 || keys[i + 1] != k) ranges[k].y = i + 1;
  }
}

void launch_ranges(FrameDev* fd, const uint32_t* keys, uint2* ranges, int n_sm, cudaStream_t s) {
  k_ranges<<<n_sm * 8, 256, 0, s>>>(fd, keys, ranges);
}

// ------------------------------------------------------------------ blend (K10)
// One block per (camera, tile) (or a persistent grid taking tiles from a
// counter); each lane owns a vertical strip of 4 pixels (lanes of a warp
// cover the tile's columns, so a warp owns a band of rows).
// Each warp walks the tile's record list on its own, 32 records at a time:
// lane l loads record l of the chunk (with the blend view the projection
// wrote for it: C, log2 opacity, box half extents), tests its opacity-aware
// box and then the ellipse itself against the warp's band.  The hits are
// the chunk's work list: compacted into consecutive shared-memory slots in
// list order (slot = the hits of the lanes below), each holding the
// band-local quadratic of the record's power in the exp2 domain,
//   log2(o) - (log2 e / 2) q(D) = [F + X (D + A' X)] + Y [(E + B' X) + C' Y],
// with (X, Y) the pixel centre relative to the band's centre (the bracket
// in X is per lane, so a pixel costs 2 FMA).  The warp walks the slots in
// order, eight records per unrolled step.  Each pixel walks them front to
// back:
//   alpha = min(0.99, 2^power), taken as 0 when the power is below
//   log2(1/255) (alpha < 1/255 is skipped: it then changes nothing);
//   stop before a Gaussian that would bring T (1 - alpha) below 1e-4;
//   C += c w, T -= w with w = alpha T;  out = C + T bg.
// A lane's 4 vertical pixels run as two pairs on the packed FP32x2 pipe
// (FFMA2/FMUL2: one issue slot for two pixels); staged coefficients are
// stored twice ({a, a}) so they feed packed operands directly.  The clamp
// to 0.99 is only applied for records whose opacity can reach it (below
// opacity 0.985 the approximated 2^power stays under 0.99): a chunk none
// of whose hits can reach it walks one record form, the others test each
// slot's bit.  A warp stops once all its pixels have; no block-wide barrier.
constexpr int BLEND_PPL = 4;                 // pixels per lane (vertical): two packed pairs
// 2^x by the hardware approximation (relative error ~2^-22; -inf -> 0).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// 1/x and sqrt(x) by the hardware approximations (relative errors ~1e-7):
// the band test below only has to stay conservative, and its slack is four
// orders of magnitude wider
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {  // a - b, round to nearest, per element
  float2 d;
  asm("{.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
constexpr int BLEND_MAX_NT = 256;
constexpr int BLEND_MAX_WARPS = BLEND_MAX_NT / 32;
constexpr float LOG2E_HALF = 0.72134752044448170368f;   // log2(e) / 2
constexpr float LOG2_MIN_ALPHA = -7.99435343685885793f;  // log2(1/255)
constexpr float LOG2_CLAMP_OPACITY = -0.02180437f;      // log2(0.985): records at or above it take the 0.99 clamp

struct BlendSmem {  // per warp, one slot per record of the current chunk's work list (in list order)
  float4 fd[BLEND_MAX_WARPS][32];   // F, F, D, D
  float4 ea[BLEND_MAX_WARPS][32];   // E, E, A', A'
  float4 bc[BLEND_MAX_WARPS][32];   // B', B', C', C'
  float4 rg[BLEND_MAX_WARPS][32];   // r, r, g, g
  float2 bl[BLEND_MAX_WARPS][32];   // b, b
  uint8_t pos[BLEND_MAX_WARPS][32];  // counting variant: the record's position in the chunk
};

__device__ __forceinline__ float2 dup2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float half_of(float2 v, int i) { return i ? v.y : v.x; }

struct PixState {
  float2 T2[2], C0[2], C1[2], C2[2];
  float thr[BLEND_PPL];  // log2(1/255) while pixel k blends, +inf once it has stopped (or is off-image)
  unsigned live;         // bit k: pixel k still blending
};

// One staged record through the lane's 4 pixels.  Returns the chunk-relative
// stop mask (bit k: pixel k stopped at this record).
template <bool CLAMP>
__device__ __forceinline__ unsigned blend_record(PixState& ps, const BlendSmem& sm, int warp, int u, float2 X2,
                                                 const float2 (&Y2)[2]) {
  const float4 s0 = sm.fd[warp][u], s1 = sm.ea[warp][u], s2 = sm.bc[warp][u], s3 = sm.rg[warp][u];
  const float2 s4 = sm.bl[warp][u];
  const float2 pa = __ffma2_rn(X2, __ffma2_rn(dup2(s1.z, s1.w), X2, dup2(s0.z, s0.w)), dup2(s0.x, s0.y));
  const float2 pb = __ffma2_rn(dup2(s2.x, s2.y), X2, dup2(s1.x, s1.y));  // E + B' X
  const float2 cq = dup2(s2.z, s2.w);
  float2 w[2], tt[2];
  bool stop = false;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float2 p = __ffma2_rn(Y2[j], __ffma2_rn(cq, Y2[j], pb), pa);
    float a0 = p.x >= ps.thr[2 * j] ? ex2_approx(p.x) : 0.f;  // alpha < 1/255 contributes nothing
    float a1 = p.y >= ps.thr[2 * j + 1] ? ex2_approx(p.y) : 0.f;
    if (CLAMP) {
      a0 = fminf(0.99f, a0);
      a1 = fminf(0.99f, a1);
    }
    w[j] = __fmul2_rn(dup2(a0, a1), ps.T2[j]);  // alpha T
    tt[j] = fsub2(ps.T2[j], w[j]);              // T (1 - alpha)
    stop |= (tt[j].x < 1e-4f) | (tt[j].y < 1e-4f);
  }
  unsigned stopped = 0;
  if (stop) {  // a pixel stops before this Gaussian: it takes nothing from it, nor after
#pragma unroll
    for (int k = 0; k < BLEND_PPL; ++k) {
      const int j = k >> 1;
      if (half_of(tt[j], k & 1) < 1e-4f) {
        ps.thr[k] = INFINITY;
        ps.live &= ~(1u << k);
        stopped |= 1u << k;
        if (k & 1) {
          w[j].y = 0.f;
          tt[j].y = ps.T2[j].y;
        } else {
          w[j].x = 0.f;
          tt[j].x = ps.T2[j].x;
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    ps.C0[j] = __ffma2_rn(dup2(s3.x, s3.y), w[j], ps.C0[j]);
    ps.C1[j] = __ffma2_rn(dup2(s3.z, s3.w), w[j], ps.C1[j]);
    ps.C2[j] = __ffma2_rn(s4, w[j], ps.C2[j]);
    ps.T2[j] = tt[j];
  }
  return stopped;
}

// A frame whose statistics nobody waits for keeps its error bits and its
// buffer needs until the host's next synchronising call reads them.
__device__ __forceinline__ void keep_frame_error(FrameDev* fd, const FrameIn* fin) {
  if (!fin->keep_err || !fd->err) return;
  atomicOr(&fd->err_sticky, fd->err);
  atomicMax(&fd->need_sticky[0], fd->n_records_need);
  atomicMax(&fd->need_sticky[1], fd->n_pairs);
}

template <bool COUNT>
__device__ __forceinline__ void blend_tile(uint32_t tile_key, BlendSmem& sm, FrameDev* __restrict__ fd,
                                           const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
                                           const Records& rec, const FrameIn* __restrict__ fin) {
  static_assert(BLEND_PPL == 4, "the packed loop handles two pairs per lane");
  const int TW = (int)fd->tile_w, TH = (int)fd->tile_h;
  uint32_t cam = 0;
  while (cam + 1 < fd->n_cams && fd->cam[cam + 1].tile_base <= tile_key) ++cam;
  const CamDev& cd = fd->cam[cam];
  const uint32_t tl = tile_key - cd.tile_base;
  const int tx = (int)(tl % (uint32_t)cd.ntx), ty = (int)(tl / (uint32_t)cd.ntx);
  const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
  const int groups = 32 / TW;                       // strips per column within a warp
  const int band = groups * BLEND_PPL;              // rows per warp
  const int lx = lane % TW, ly0 = warp * band + (lane / TW) * BLEND_PPL;
  const int px = tx * TW + lx, py0 = ty * TH + ly0;
  // origin of the quadratic: the centre of the warp's band (|X| <= TW/2,
  // |Y| <= band/2 whatever the tile height, which bounds the float32
  // rounding of the expanded power)
  const float ox = (float)(tx * TW) + 0.5f * (float)TW, oy = (float)(ty * TH + warp * band) + 0.5f * (float)band;
  const float X = ((float)px + 0.5f) - ox;
  const float Y0 = ((float)py0 + 0.5f) - oy;
  const float wx0 = ((float)(tx * TW) + 0.5f) - ox, wx1 = wx0 + (float)(TW - 1);
  const float wy0 = ((float)(ty * TH + warp * band) + 0.5f) - oy, wy1 = wy0 + (float)(band - 1);
  const uint2 rg = ranges[tile_key];
  const float2 X2 = dup2(X, X);
  const float2 Y2[2] = {dup2(Y0, Y0 + 1.f), dup2(Y0 + 2.f, Y0 + 3.f)};
  PixState ps;
  ps.live = 0;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    ps.T2[j] = dup2(1.f, 1.f);
    ps.C0[j] = ps.C1[j] = ps.C2[j] = dup2(0.f, 0.f);
  }
#pragma unroll
  for (int k = 0; k < BLEND_PPL; ++k) {
    const bool in = px < cd.W && py0 + k < cd.H;
    ps.live |= (in ? 1u : 0u) << k;
    ps.thr[k] = in ? LOG2_MIN_ALPHA : INFINITY;
  }
  uint32_t n_walk = 0, n_issued = 0;  // counting variant only
  const unsigned lt_lanes = (1u << lane) - 1u;
  for (uint32_t b = rg.x; b < rg.y; b += 32u) {
    if (!__any_sync(0xffffffffu, ps.live != 0)) break;  // every pixel of the warp has stopped
    const uint32_t idx = b + (uint32_t)lane;
    bool hit = false;
    uint32_t r = 0;
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f), c = g, cl = g;
    if (idx < rg.y) {
      r = vals[idx];
      g = rec.geo[r];  // mean x, mean y, A, B
      c = rec.aux[r];  // C, log2(opacity), box half-width, box half-height
      cl = rec.col[r];  // (with the geometry: one round trip for all three, hit or not)
      const float mxl = g.x - ox, myl = g.y - oy;
      const float A = g.z, B = g.w, Cc = c.x;
      hit = !(mxl + c.z < wx0 || mxl - c.z > wx1 || myl + c.w < wy0 || myl - c.w > wy1);  // box meets the band
      if (hit) {  // the ellipse itself: its x-extent over the band's rows against the band's columns
        // on the row dy (from the mean) the ellipse spans dx = (-B dy +- sqrt(det) sqrt(ey^2 - dy^2)) / A;
        // its right- and leftmost points lie on dy = -+B ex / C, clamped to the band's rows
        const float ya = fmaxf(wy0 - myl, -c.w), yb = fminf(wy1 - myl, c.w);
        const float iA = rcp_approx(A), sd = sqrt_approx(fmaxf(0.f, A * Cc - B * B)) * iA;
        const float bxc = B * c.z * rcp_approx(Cc), h2 = c.w * c.w, bA = B * iA;
        const float dr = fminf(fmaxf(-bxc, ya), yb), dl = fminf(fmaxf(bxc, ya), yb);
        const float xr = mxl - bA * dr + sd * sqrt_approx(fmaxf(0.f, h2 - dr * dr));
        const float xl = mxl - bA * dl - sd * sqrt_approx(fmaxf(0.f, h2 - dl * dl));
        // float32 rounding and the approximations (the box's tau is already
        // enlarged); a record kept in excess only evaluates below 1/255
        const float slack = 1e-3f * (c.z + 1.f);
        hit = xr + slack >= wx0 && xl - slack <= wx1;
      }
    }
    // the chunk's work list: the hits, compacted into slots 0 .. nh-1 in list order
    const unsigned hm = __ballot_sync(0xffffffffu, hit);
    const uint32_t nh = (uint32_t)__popc(hm), slot = (uint32_t)__popc(hm & lt_lanes);
    bool clamp = false;
    if (hit) {
      const float mxl = g.x - ox, myl = g.y - oy;
      const float A = g.z, B = g.w, Cc = c.x;
      const float q0 = A * mxl * mxl + 2.f * B * mxl * myl + Cc * myl * myl;
      const float F = c.y - LOG2E_HALF * q0;
      const float D = 2.f * LOG2E_HALF * (A * mxl + B * myl);
      const float E = 2.f * LOG2E_HALF * (B * mxl + Cc * myl);
      const float Ap = -LOG2E_HALF * A, Bp = -2.f * LOG2E_HALF * B, Cp = -LOG2E_HALF * Cc;
      sm.fd[warp][slot] = make_float4(F, F, D, D);
      sm.ea[warp][slot] = make_float4(E, E, Ap, Ap);
      sm.bc[warp][slot] = make_float4(Bp, Bp, Cp, Cp);
      sm.rg[warp][slot] = make_float4(cl.x, cl.x, cl.y, cl.y);
      sm.bl[warp][slot] = make_float2(cl.z, cl.z);
      if (COUNT) sm.pos[warp][slot] = (uint8_t)lane;
      clamp = c.y >= LOG2_CLAMP_OPACITY;
    }
    const unsigned cmask = __reduce_or_sync(0xffffffffu, clamp ? 1u << slot : 0u);  // by slot
    __syncwarp();
    const uint32_t cnt = min(32u, rg.y - b);
    if (COUNT) {
      n_walk += (uint32_t)__popc(ps.live) * cnt;
      n_issued += nh * BLEND_PPL;
    }
    if (cmask == 0u) {  // no record of the list reaches the 0.99 clamp
      // (unrolled: consecutive records' independent loads and quadratics
      // interleave with the previous one's dependent chain)
#pragma unroll 8
      for (uint32_t u = 0; u < nh; ++u) {
        const unsigned st = blend_record<false>(ps, sm, warp, (int)u, X2, Y2);
        if (COUNT && st) n_walk -= (uint32_t)__popc(st) * (cnt - 1u - (uint32_t)sm.pos[warp][u]);
      }
    } else {
      for (uint32_t u = 0; u < nh; ++u) {
        const unsigned st = ((cmask >> u) & 1u) ? blend_record<true>(ps, sm, warp, (int)u, X2, Y2)
                                                : blend_record<false>(ps, sm, warp, (int)u, X2, Y2);
        if (COUNT && st) n_walk -= (uint32_t)__popc(st) * (cnt - 1u - (uint32_t)sm.pos[warp][u]);
      }
    }
    __syncwarp();  // the slots are rewritten by the next chunk
  }
  if (fin->out_format == 0) {
    float* out = reinterpret_cast<float*>(fin->out_rgb[cam]);
#pragma unroll
    for (int k = 0; k < BLEND_PPL; ++k) {
      const int py = py0 + k;
      if (px >= cd.W || py >= cd.H) continue;
      const size_t p = ((size_t)py * cd.W + px) * 3;
      const float T = half_of(ps.T2[k >> 1], k & 1);
      out[p + 0] = half_of(ps.C0[k >> 1], k & 1) + T * fin->bg[0];
      out[p + 1] = half_of(ps.C1[k >> 1], k & 1) + T * fin->bg[1];
      out[p + 2] = half_of(ps.C2[k >> 1], k & 1) + T * fin->bg[2];
    }
  } else {  // RGBA8: round-to-nearest-even of 255 x clamp(colour), alpha 1 - T
    uchar4* out = reinterpret_cast<uchar4*>(fin->out_rgb[cam]);
#pragma unroll
    for (int k = 0; k < BLEND_PPL; ++k) {
      const int py = py0 + k;
      if (px >= cd.W || py >= cd.H) continue;
      const float T = half_of(ps.T2[k >> 1], k & 1);
      out[(size_t)py * cd.W + px] = make_uchar4(
          (unsigned char)__float2uint_rn(__saturatef(half_of(ps.C0[k >> 1], k & 1) + T * fin->bg[0]) * 255.f),
          (unsigned char)__float2uint_rn(__saturatef(half_of(ps.C1[k >> 1], k & 1) + T * fin->bg[1]) * 255.f),
          (unsigned char)__float2uint_rn(__saturatef(half_of(ps.C2[k >> 1], k & 1) + T * fin->bg[2]) * 255.f),
          (unsigned char)__float2uint_rn(__saturatef(1.f - T) * 255.f));
    }
  }
  float* outT = reinterpret_cast<float*>(fin->out_T[cam]);
  if (outT) {
#pragma unroll
    for (int k = 0; k < BLEND_PPL; ++k) {
      const int py = py0 + k;
      if (px < cd.W && py < cd.H) outT[(size_t)py * cd.W + px] = half_of(ps.T2[k >> 1], k & 1);
    }
  }
  if (COUNT) {
    const uint32_t w = __reduce_add_sync(0xffffffffu, n_walk), i = __reduce_add_sync(0xffffffffu, n_issued);
    if (lane == 0) {
      atomicAdd(&fd->blend_work[0], (unsigned long long)w);
      atomicAdd(&fd->blend_work[1], (unsigned long long)i);
    }
  }
}

// One block per tile of every camera.
template <bool COUNT>
__global__ void __launch_bounds__(BLEND_MAX_NT, 4) k_blend(FrameDev* __restrict__ fd, const uint2* __restrict__ ranges,
                                                        const uint32_t* __restrict__ vals, Records rec,
                                                        const FrameIn* __restrict__ fin) {
  __shared__ BlendSmem sm;
  if (blockIdx.x == 0 && threadIdx.x == 0) keep_frame_error(fd, fin);
  blend_tile<COUNT>(blockIdx.x, sm, fd, ranges, vals, rec, fin);
}

// Persistent form: a fixed grid (blocks per SM x SMs) whose blocks take the
// tiles of all cameras - of every viewer in a batched frame - from one
// counter, so long and short tiles balance across the machine.
template <bool COUNT>
__global__ void __launch_bounds__(BLEND_MAX_NT, 4) k_blend_persistent(FrameDev* __restrict__ fd,
                                                                   const uint2* __restrict__ ranges,
                                                                   const uint32_t* __restrict__ vals, Records rec,
                                                                   const FrameIn* __restrict__ fin) {
  __shared__ BlendSmem sm;
  __shared__ uint32_t s_tile;
  if (blockIdx.x == 0 && threadIdx.x == 0) keep_frame_error(fd, fin);
  const uint32_t total = fd->total_tiles;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_tile = atomicAdd(&fd->ctr[SLOT_BLEND], 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= total) break;
    blend_tile<COUNT>(tile, sm, fd, ranges, vals, rec, fin);
  }
}

void launch_blend(FrameDev* fd, const uint2* ranges, const uint32_t* vals, Records rec, const FrameIn* fin,
                  uint32_t total_tiles, uint32_t tile_threads, uint32_t blocks_per_sm, bool count, int n_sm,
                  cudaStream_t s) {
  const uint32_t nt = tile_threads / BLEND_PPL, grid = n_sm * blocks_per_sm;
  if (blocks_per_sm == 0) {
    if (count)
      k_blend<true><<<total_tiles, nt, 0, s>>>(fd, ranges, vals, rec, fin);
    else
      k_blend<false><<<total_tiles, nt, 0, s>>>(fd, ranges, vals, rec, fin);
  } else {
    if (count)
      k_blend_persistent<true><<<grid, nt, 0, s>>>(fd, ranges, vals, rec, fin);
    else
      k_blend_persistent<false><<<grid, nt, 0, s>>>(fd, ranges, vals, rec, fin);
  }
}

}  // namespace gsc
