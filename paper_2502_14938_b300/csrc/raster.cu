// Splatting back half: pair offsets (K6), key generation (K7), tile ranges
// (K9) and front-to-back alpha blending (K10).  Sec. 3.1 (tile
// rasterisation), Sec. 6 (opacity-aware extent, exact tile coverage).
#include "gsc_internal.cuh"

namespace gsc {

// ------------------------------------------------------------------ scan (K6)
// Exclusive prefix sum of cnt[order[i]] (or cnt[i] without order) for
// i < *n_ptr, one pass with a decoupled look-back; *total_out = the sum.
constexpr int SCAN_NT = 256;
constexpr int SCAN_IPT = 16;
constexpr int SCAN_TILE = SCAN_NT * SCAN_IPT;

__global__ void __launch_bounds__(SCAN_NT) k_scan(const uint32_t* __restrict__ cnt, const uint32_t* __restrict__ order,
                                                  const uint32_t* __restrict__ n_ptr, uint32_t* __restrict__ out,
                                                  uint32_t* total_out, unsigned long long* status, FrameDev* fd,
                                                  int slot) {
  __shared__ uint32_t s_warp[SCAN_NT / 32 + 1];
  __shared__ uint32_t s_base;
  __shared__ uint32_t s_tile;
  const uint32_t n = *n_ptr;
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
    if (threadIdx.x == 0) {
      unsigned long long* w = status + t;
      uint32_t pre = 0;
      if (t == 0) {
        st_relaxed_u64(w, lb_pack(epoch, 2u, tot));
      } else {
        st_relaxed_u64(w, lb_pack(epoch, 1u, tot));
        pre = lb_exclusive(status, 1, t, epoch, spin, &fd->err);
        st_relaxed_u64(w, lb_pack(epoch, 2u, pre + tot));
      }
      s_base = pre;
      if (t == ntiles - 1) *total_out = pre + tot;
    }
    __syncthreads();
    uint32_t run = s_base + ex;
#pragma unroll
    for (int u = 0; u < SCAN_IPT; ++u) {
      const uint32_t i = i0 + u;
      if (i < n) out[i] = run;
      run += v[u];
    }
    __syncthreads();
  }
}

void launch_scan_u32(const uint32_t* cnt, const uint32_t* order, const uint32_t* n_ptr, uint32_t* out,
                     uint32_t* total_out, unsigned long long* status, FrameDev* fd, int slot, int n_sm,
                     cudaStream_t s) {
  k_scan<<<n_sm * 2, SCAN_NT, 0, s>>>(cnt, order, n_ptr, out, total_out, status, fd, slot);
}

// ------------------------------------------------------------------ key generation (K7)
// For the i-th record in depth order, emit (tile_base(camera) + tile, record)
// at offs[i] .. offs[i] + cnt - 1, tiles in row-major order of the exact
// coverage.  Pairs beyond the capacity are not written and flag an overflow.
// A record covering at most KG_SMALL tiles is emitted by its own thread.
// Larger ones (near-camera Gaussians, up to thousands of tiles) cluster at
// the front of the depth order, so they go to a work list that a second
// kernel spreads over all warps, one record per warp: lane l computes the
// range of tile row ty0 + l (32 rows at once), a warp scan gives each row's
// offset, and the lanes write the tiles of each row.  The float32 row ranges
// are the ones the count pass used, so the pairs and their order are the same.
constexpr uint32_t KG_SMALL = 32;

__global__ void __launch_bounds__(256) k_keygen(FrameDev* __restrict__ fd, Records rec, const uint32_t* __restrict__ order,
                                                const uint32_t* __restrict__ offs, uint32_t* __restrict__ pkeys,
                                                uint32_t* __restrict__ pvals, uint32_t cap, uint32_t* __restrict__ big) {
  const uint32_t n = fd->n_valid;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const uint32_t np = fd->n_pairs;
    fd->n_pairs_used = np < cap ? np : cap;
    if (np > cap) atomicOr(&fd->err, ERR_PAIR_OVERFLOW);
  }
  const int TW = (int)fd->tile_w, TH = (int)fd->tile_h;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t r = order[i];
    const uint32_t c = rec.cnt[r];
    if (c > KG_SMALL) {
      big[atomicAdd(&fd->n_big, 1u)] = i;
      continue;
    }
    uint32_t o = offs[i];
    const float4 g = rec.geo[r];
    const float4 cp = rec.cop[r];
    const CamDev& cd = fd->cam[__float_as_uint(rec.col[r].w) & 0xFFFFu];
    const uint32_t tb = cd.tile_base;
    cover_tiles_f32(g.x, g.y, g.z, g.w, cp.x, cp.z, cd.W, cd.H, TW, TH, [&](int tile) {
      if (o < cap) {
        pkeys[o] = tb + (uint32_t)tile;
        pvals[o] = r;
      }
      ++o;
    });
  }
}

__global__ void __launch_bounds__(256) k_keygen_big(FrameDev* __restrict__ fd, Records rec,
                                                    const uint32_t* __restrict__ order, const uint32_t* __restrict__ offs,
                                                    uint32_t* __restrict__ pkeys, uint32_t* __restrict__ pvals,
                                                    uint32_t cap, const uint32_t* __restrict__ big) {
  const uint32_t nb = fd->n_big;
  const int TW = (int)fd->tile_w, TH = (int)fd->tile_h;
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
        for (uint32_t u = lane; u < l; u += 32u) {
          const uint32_t oi = o + ex + u;
          if (oi < cap) {
            pkeys[oi] = kb + u;
            pvals[oi] = r;
          }
        }
      }
      o += chunk;
    }
  }
}

void launch_keygen(FrameDev* fd, Records rec, const uint32_t* order, const uint32_t* offs, uint32_t* pkeys,
                   uint32_t* pvals, uint32_t cap, uint32_t* big, int n_sm, cudaStream_t s) {
  k_keygen<<<n_sm * 8, 256, 0, s>>>(fd, rec, order, offs, pkeys, pvals, cap, big);
  k_keygen_big<<<n_sm * 4, 256, 0, s>>>(fd, rec, order, offs, pkeys, pvals, cap, big);
}

// ------------------------------------------------------------------ tile ranges (K9)
__global__ void k_ranges(const FrameDev* __restrict__ fd, const uint32_t* __restrict__ keys, uint2* __restrict__ ranges) {
  const uint32_t n = fd->n_pairs_used;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t k = keys[i];
    if (i == 0 || keys[i - 1] != k) ranges[k].x = i;
    if (i == n - 1 || keys[i + 1] != k) ranges[k].y = i + 1;
  }
}

void launch_ranges(FrameDev* fd, const uint32_t* keys, uint2* ranges, int n_sm, cudaStream_t s) {
  k_ranges<<<n_sm * 8, 256, 0, s>>>(fd, keys, ranges);
}

// ------------------------------------------------------------------ blend (K10)
// One block per (camera, tile), one thread per pixel; warp w owns an 8x4
// block of pixels.  The tile's records are staged into shared memory one
// batch at a time, each turned into the tile-local quadratic of its power in
// the exp2 domain,
//   log2(o) - (log2 e / 2) q(D) = F + X (D + A' X + B' Y) + Y (E + C' Y),
// with (X, Y) the pixel centre relative to the tile centre, plus the
// Gaussian's opacity-aware bounding box.  Each pixel then walks the batch
// front to back:
//   skip if the power is below log2(1/255) (alpha < 1/255);
//   alpha = min(0.99, 2^power);
//   stop before a Gaussian that would bring T (1 - alpha) below 1e-4;
//   C += c alpha T, T *= 1 - alpha;  out = C + T bg.
// A warp skips a Gaussian whose box misses its 8x4 pixels, and skips the
// whole batch once its pixels are finished; the block stops once all are.
constexpr int BLEND_MAX_NT = 256;
constexpr float LOG2E_HALF = 0.72134752044448170368f;  // log2(e) / 2
constexpr float LOG2_MIN_ALPHA = -7.99435343685885793f;  // log2(1/255)

__global__ void __launch_bounds__(BLEND_MAX_NT) k_blend(const FrameDev* __restrict__ fd, const uint2* __restrict__ ranges,
                                                        const uint32_t* __restrict__ vals, Records rec,
                                                        const FrameIn* __restrict__ fin) {
  __shared__ float4 s_q0[BLEND_MAX_NT];   // F, D, E, A'
  __shared__ float4 s_q1[BLEND_MAX_NT];   // B', C', r, g
  __shared__ float4 s_bb[BLEND_MAX_NT];   // b, xmin, xmax, ymin
  __shared__ float s_ymax[BLEND_MAX_NT];
  const uint32_t tile_key = blockIdx.x;
  const int TW = (int)fd->tile_w, TH = (int)fd->tile_h;
  const int nt = TW * TH;
  uint32_t cam = 0;
  while (cam + 1 < fd->n_cams && fd->cam[cam + 1].tile_base <= tile_key) ++cam;
  const CamDev& cd = fd->cam[cam];
  const uint32_t tl = tile_key - cd.tile_base;
  const int tx = (int)(tl % (uint32_t)cd.ntx), ty = (int)(tl / (uint32_t)cd.ntx);
  // warp -> 8x4 pixel block, lane -> pixel
  const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
  const int wpr = TW >> 3;  // warp blocks per tile row
  const int bx = (warp % wpr) * 8, by = (warp / wpr) * 4;
  const int lx = bx + (lane & 7), ly = by + (lane >> 3);
  const int px = tx * TW + lx, py = ty * TH + ly;
  const bool inside = px < cd.W && py < cd.H;
  const float ox = (float)(tx * TW) + 0.5f * (float)TW, oy = (float)(ty * TH) + 0.5f * (float)TH;
  const float X = ((float)px + 0.5f) - ox, Y = ((float)py + 0.5f) - oy;
  // the warp's pixel-centre box in tile-local coordinates
  const float wx0 = ((float)(tx * TW + bx) + 0.5f) - ox, wx1 = wx0 + 7.f;
  const float wy0 = ((float)(ty * TH + by) + 0.5f) - oy, wy1 = wy0 + 3.f;
  const uint2 rg = ranges[tile_key];
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  bool done = !inside;
  for (uint32_t b = rg.x; b < rg.y; b += (uint32_t)nt) {
    if (__syncthreads_count(done) == nt) break;
    const uint32_t idx = b + threadIdx.x;
    if (idx < rg.y) {
      const uint32_t r = vals[idx];
      const float4 g = rec.geo[r];   // mean x, mean y, A, B
      const float4 c = rec.cop[r];   // C, opacity, tau, depth
      const float4 cl = rec.col[r];
      const float mxl = g.x - ox, myl = g.y - oy;
      const float A = g.z, B = g.w, Cc = c.x;
      const float q0 = A * mxl * mxl + 2.f * B * mxl * myl + Cc * myl * myl;
      s_q0[threadIdx.x] = make_float4(__log2f(c.y) - LOG2E_HALF * q0, 2.f * LOG2E_HALF * (A * mxl + B * myl),
                                      2.f * LOG2E_HALF * (B * mxl + Cc * myl), -LOG2E_HALF * A);
      s_q1[threadIdx.x] = make_float4(-2.f * LOG2E_HALF * B, -LOG2E_HALF * Cc, cl.x, cl.y);
      const float idet = 1.f / (A * Cc - B * B);
      const float ex = sqrtf(c.z * Cc * idet), ey = sqrtf(c.z * A * idet);
      s_bb[threadIdx.x] = make_float4(cl.z, mxl - ex, mxl + ex, myl - ey);
      s_ymax[threadIdx.x] = myl + ey;
    }
    __syncthreads();
    const int cnt = min(nt, (int)(rg.y - b));
    if (__all_sync(0xffffffffu, done)) continue;
    for (int u = 0; u < cnt; ++u) {
      const float4 bb = s_bb[u];
      if (bb.z < wx0 || bb.y > wx1 || bb.w > wy1 || s_ymax[u] < wy0) continue;  // box misses the warp
      if (done) continue;
      const float4 q0 = s_q0[u];
      const float4 q1 = s_q1[u];
      const float t1 = fmaf(q0.w, X, fmaf(q1.x, Y, q0.y));
      const float t2 = fmaf(q1.y, Y, q0.z);
      const float p = fmaf(t1, X, fmaf(t2, Y, q0.x));
      if (p < LOG2_MIN_ALPHA) continue;
      const float alpha = fminf(0.99f, exp2f(p));
      const float tt = fmaf(-T, alpha, T);
      if (tt < 1e-4f) {
        done = true;
        continue;
      }
      const float w = alpha * T;
      C0 = fmaf(q1.z, w, C0);
      C1 = fmaf(q1.w, w, C1);
      C2 = fmaf(bb.x, w, C2);
      T = tt;
    }
  }
  if (inside) {
    float* out = reinterpret_cast<float*>(fin->out_rgb[cam]);
    const size_t p = ((size_t)py * cd.W + px) * 3;
    out[p + 0] = C0 + T * fin->bg[0];
    out[p + 1] = C1 + T * fin->bg[1];
    out[p + 2] = C2 + T * fin->bg[2];
    if (fin->out_T[cam]) reinterpret_cast<float*>(fin->out_T[cam])[(size_t)py * cd.W + px] = T;
  }
}

void launch_blend(FrameDev* fd, const uint2* ranges, const uint32_t* vals, Records rec, const FrameIn* fin,
                  uint32_t total_tiles, uint32_t tile_threads, cudaStream_t s) {
  k_blend<<<total_tiles, tile_threads, 0, s>>>(fd, ranges, vals, rec, fin);
}

}  // namespace gsc
