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
__global__ void __launch_bounds__(256) k_keygen(FrameDev* __restrict__ fd, Records rec, const uint32_t* __restrict__ order,
                                                const uint32_t* __restrict__ offs, uint32_t* __restrict__ pkeys,
                                                uint32_t* __restrict__ pvals, uint32_t cap) {
  const uint32_t n = fd->n_valid;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const uint32_t np = fd->n_pairs;
    fd->n_pairs_used = np < cap ? np : cap;
    if (np > cap) atomicOr(&fd->err, ERR_PAIR_OVERFLOW);
  }
  const int TW = (int)fd->tile_w, TH = (int)fd->tile_h;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t r = order[i];
    uint32_t o = offs[i];
    const float4 g = rec.geo[r];
    const float4 c = rec.cop[r];
    const uint32_t cam = __float_as_uint(rec.col[r].w) & 0xFFFFu;
    const CamDev& cd = fd->cam[cam];
    const uint32_t tb = cd.tile_base;
    cover_tiles_f32(g.x, g.y, g.z, g.w, c.x, c.z, cd.W, cd.H, TW, TH, [&](int tile) {
      if (o < cap) {
        pkeys[o] = tb + (uint32_t)tile;
        pvals[o] = r;
      }
      ++o;
    });
  }
}

void launch_keygen(FrameDev* fd, Records rec, const uint32_t* order, const uint32_t* offs, uint32_t* pkeys,
                   uint32_t* pvals, uint32_t cap, int n_sm, cudaStream_t s) {
  k_keygen<<<n_sm * 8, 256, 0, s>>>(fd, rec, order, offs, pkeys, pvals, cap);
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
// One block per (camera, tile), one thread per pixel.  The tile's records
// are staged into shared memory one batch at a time; each pixel walks them
// front to back:
//   D = pixel centre - mean, power = -(A Dx^2 + C Dy^2)/2 - B Dx Dy,
//   alpha = min(0.99, o exp(power)), skipped if < 1/255;
//   stop before a Gaussian that would bring T (1 - alpha) below 1e-4;
//   C += c alpha T, T *= 1 - alpha;  out = C + T bg.
// A warp whose pixels are all finished skips the batch; the block stops
// once every pixel is finished.
constexpr int BLEND_MAX_NT = 256;

__global__ void __launch_bounds__(BLEND_MAX_NT) k_blend(const FrameDev* __restrict__ fd, const uint2* __restrict__ ranges,
                                                        const uint32_t* __restrict__ vals, Records rec,
                                                        const FrameIn* __restrict__ fin) {
  __shared__ float4 s_geo[BLEND_MAX_NT];
  __shared__ float2 s_co[BLEND_MAX_NT];
  __shared__ float4 s_col[BLEND_MAX_NT];
  const uint32_t tile_key = blockIdx.x;
  const int TW = (int)fd->tile_w, TH = (int)fd->tile_h;
  const int nt = TW * TH;
  uint32_t cam = 0;
  while (cam + 1 < fd->n_cams && fd->cam[cam + 1].tile_base <= tile_key) ++cam;
  const CamDev& cd = fd->cam[cam];
  const uint32_t tl = tile_key - cd.tile_base;
  const int tx = (int)(tl % (uint32_t)cd.ntx), ty = (int)(tl / (uint32_t)cd.ntx);
  const int px = tx * TW + (int)threadIdx.x % TW;
  const int py = ty * TH + (int)threadIdx.x / TW;
  const bool inside = px < cd.W && py < cd.H;
  const float X = (float)px + 0.5f, Y = (float)py + 0.5f;
  const uint2 rg = ranges[tile_key];
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  bool done = !inside;
  for (uint32_t b = rg.x; b < rg.y; b += (uint32_t)nt) {
    if (__syncthreads_count(done) == nt) break;
    const uint32_t idx = b + threadIdx.x;
    if (idx < rg.y) {
      const uint32_t r = vals[idx];
      s_geo[threadIdx.x] = rec.geo[r];
      const float4 c = rec.cop[r];
      s_co[threadIdx.x] = make_float2(c.x, c.y);
      s_col[threadIdx.x] = rec.col[r];
    }
    __syncthreads();
    const int cnt = min(nt, (int)(rg.y - b));
    if (!__all_sync(0xffffffffu, done)) {
      for (int u = 0; u < cnt && !done; ++u) {
        const float4 g = s_geo[u];
        const float2 co = s_co[u];
        const float dx = X - g.x, dy = Y - g.y;
        const float power = -0.5f * (g.z * dx * dx + co.x * dy * dy) - g.w * dx * dy;
        const float alpha = fminf(0.99f, co.y * __expf(power));
        if (alpha < (1.0f / 255.0f)) continue;
        const float tt = T * (1.f - alpha);
        if (tt < 1e-4f) {
          done = true;
          break;
        }
        const float4 cl = s_col[u];
        const float w = alpha * T;
        C0 += cl.x * w;
        C1 += cl.y * w;
        C2 += cl.z * w;
        T = tt;
      }
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
