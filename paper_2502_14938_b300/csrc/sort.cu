// LSD radix sort of (uint32 key, uint32 value) pairs, 8- or 9-bit digits,
// "onesweep" style: one kernel computes the digit histograms of every pass
// (or the key producer accumulates them);
// each pass is then one kernel in which a block ranks a tile of keys
// (warp match + per-warp digit counters, stable), obtains its per-digit
// global offsets by a decoupled look-back over the preceding tiles, and
// scatters through shared memory so that global writes are mostly
// contiguous.  Stable, so sorting records by depth and then pairs by tile
// yields the (tile, depth, Gaussian id) order of the key definition.
// Tiles are taken from an atomic counter in increasing order: a block only
// waits on tiles already held by running blocks, and every wait is bounded.
// The grid is two blocks per SM: when every tile of a pass is in flight at
// once, tile t walks back over ~t/16 aggregate windows and the look-back
// traffic grows with the square of the tiles in flight; fewer resident
// blocks let earlier tiles finish their prefixes first (measured: 4 or 3
// blocks per SM and a 16- or 32-word window were slower).  4096-key tiles
// are ranked by 512 threads (16 warps of 8 keys each: half the serial
// match rounds of 256 threads x 16 keys), 2048-key tiles by 512 threads of
// 4 keys (1024 threads of 4 keys for 4096-key tiles were slower).
#include "gsc_internal.cuh"

namespace gsc {


__global__ void __launch_bounds__(256) k_sort_hist(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ n_ptr,
                                                   int npass, int drop_invalid, uint32_t* __restrict__ hist,
                                                   uint32_t* n_valid_out) {
  __shared__ uint32_t s_h[4][256];
  for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) (&s_h[0][0])[i] = 0;
  __syncthreads();
  const uint32_t n = *n_ptr;
  uint32_t nv = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t k = keys[i];
    if (drop_invalid && k == INVALID_KEY) continue;
    ++nv;
    for (int p = 0; p < npass; ++p) atomicAdd(&s_h[p][(k >> (8 * p)) & 0xFFu], 1u);
  }
  __syncthreads();
  for (int p = 0; p < npass; ++p)
    for (int d = threadIdx.x; d < 256; d += blockDim.x)
      if (s_h[p][d]) atomicAdd(&hist[p * 256 + d], s_h[p][d]);
  if (n_valid_out) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nv += __shfl_xor_sync(0xffffffffu, nv, o);
    if ((threadIdx.x & 31) == 0 && nv) atomicAdd(n_valid_out, nv);
  }
}

// NT threads per block (NT / 32 warps each ranking 32 x IPT keys), tiles of
// NT x IPT keys; the keys and values of a tile are staged in dynamic shared
// memory.  Digits of DB bits (8: 256 digits, 9: 512); threads 0..2^DB - 1
// own one digit each for the histograms, scans and the look-back (digit
// status words at a stride of 2^DB per tile).  Optional, all read on the
// device: key_sub (subtracted from every kept key as it is read), run_if
// (the pass runs only if *run_if != 0) and use_alt (if *use_alt != 0 the
// output goes to kout_alt / vout_alt).
template <int NT, int IPT, int DB = 8>
__global__ void __launch_bounds__(NT, 2) k_sort_pass(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                  uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                  const uint32_t* __restrict__ n_ptr, int shift,
                                                  const uint32_t* __restrict__ hist_p, int drop_invalid,
                                                  unsigned long long* status, FrameDev* fd, int slot,
                                                  const uint32_t* __restrict__ key_sub, const uint32_t* __restrict__ run_if,
                                                  uint32_t* __restrict__ kout_alt, uint32_t* __restrict__ vout_alt,
                                                  const uint32_t* __restrict__ use_alt) {
  constexpr int TILE = NT * IPT, WARPS = NT / 32, NDIG = 1 << DB;
  constexpr uint32_t DMASK = NDIG - 1;
  static_assert(NT >= NDIG, "one thread per digit");
  __shared__ uint32_t s_gbase[NDIG];
  __shared__ uint32_t s_whist[WARPS][NDIG];
  __shared__ uint32_t s_dstart[NDIG];
  __shared__ uint32_t s_gofs[NDIG];
  __shared__ uint32_t s_warp[NT / 32 + 1];
  __shared__ uint32_t s_tile;
  extern __shared__ uint32_t s_kv[];  // keys [TILE], values [TILE]
  uint32_t* s_keys = s_kv;
  uint32_t* s_vals = s_kv + TILE;

  if (run_if && *run_if == 0u) return;
  if (use_alt && *use_alt != 0u) {
    kout = kout_alt;
    vout = vout_alt;
  }
  const uint32_t ksub = key_sub ? *key_sub : 0u;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const bool dig = tid < (uint32_t)NDIG;
  {
    uint32_t tot;
    const uint32_t g = block_exclusive_scan<NT>(dig ? hist_p[tid] : 0u, s_warp, &tot);
    if (dig) s_gbase[tid] = g;
  }
  const uint32_t n = *n_ptr;
  const uint32_t ntiles = (n + TILE - 1) / TILE;
  const uint32_t epoch = fd->frame * 64u + (uint32_t)slot;
  const uint32_t spin = fd->spin_limit;
  const uint32_t lt_mask = (1u << lane) - 1u;

  for (;;) {
    if (tid == 0) s_tile = atomicAdd(&fd->ctr[slot], 1u);
    for (int i = tid; i < WARPS * NDIG; i += NT) (&s_whist[0][0])[i] = 0;
    __syncthreads();
    const uint32_t t = s_tile;
    if (t >= ntiles) break;
    const uint32_t base = t * TILE + warp * 32u * IPT;
    uint32_t key[IPT], val[IPT], rank[IPT];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      const uint32_t idx = base + (uint32_t)i * 32u + lane;
      bool valid = idx < n;
      uint32_t k = valid ? kin[idx] : INVALID_KEY;
      if (drop_invalid && k == INVALID_KEY) valid = false;
      if (valid) k -= ksub;
      key[i] = valid ? k : INVALID_KEY;
      val[i] = valid ? (vin ? vin[idx] : idx) : 0u;
      const uint32_t d = (k >> shift) & DMASK;
      const uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : 0x1000u);
      uint32_t pre = 0;
      if (valid) pre = s_whist[warp][d];
      rank[i] = valid ? pre + (uint32_t)__popc(peers & lt_mask) : 0xFFFFFFFFu;
      __syncwarp();
      if (valid && (peers & lt_mask) == 0) s_whist[warp][d] = pre + (uint32_t)__popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // per digit: warp-exclusive offsets, tile total
    uint32_t tot_d = 0;
    if (dig) {
      const uint32_t d = tid;
#pragma unroll
      for (int w = 0; w < WARPS; ++w) {
        const uint32_t c = s_whist[w][d];
        s_whist[w][d] = tot_d;
        tot_d += c;
      }
    }
    if (dig)  // publish this tile's counts before the block scan
      st_relaxed_u64(status + (size_t)t * NDIG + tid, lb_pack(epoch, t == 0 ? 2u : 1u, tot_d));
    uint32_t tile_total;
    {
      const uint32_t ds = block_exclusive_scan<NT>(tot_d, s_warp, &tile_total);
      if (dig) s_dstart[tid] = ds;
    }
    if (dig) {
      const uint32_t d = tid;
      uint32_t pre = 0;
      if (t > 0) {
        pre = lb_exclusive(status + d, NDIG, t, epoch, spin, &fd->err);
        st_relaxed_u64(status + (size_t)t * NDIG + d, lb_pack(epoch, 2u, pre + tot_d));
      }
      s_gofs[d] = s_gbase[d] + pre;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      if (rank[i] == 0xFFFFFFFFu) continue;
      const uint32_t d = (key[i] >> shift) & DMASK;
      const uint32_t p = s_dstart[d] + s_whist[warp][d] + rank[i];
      s_keys[p] = key[i];
      s_vals[p] = val[i];
    }
    __syncthreads();
    for (uint32_t p = tid; p < tile_total; p += NT) {
      const uint32_t k = s_keys[p];
      const uint32_t d = (k >> shift) & DMASK;
      const uint32_t o = s_gofs[d] + (p - s_dstart[d]);
      if (!GSC_IN_BOUNDS(o, n, &fd->err)) continue;
      kout[o] = k;
      vout[o] = s_vals[p];
    }
    __syncthreads();
  }
}

template <int NT, int IPT, int DB = 8>
void sort_pass(int blocks, cudaStream_t s, const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout,
               const uint32_t* n_ptr, int shift, const uint32_t* hist_p, int drop_invalid, unsigned long long* status,
               FrameDev* fd, int slot, const uint32_t* key_sub = nullptr, const uint32_t* run_if = nullptr,
               uint32_t* kout_alt = nullptr, uint32_t* vout_alt = nullptr, const uint32_t* use_alt = nullptr) {
  k_sort_pass<NT, IPT, DB><<<blocks, NT, 2 * NT * IPT * sizeof(uint32_t), s>>>(
      kin, vin, kout, vout, n_ptr, shift, hist_p, drop_invalid, status, fd, slot, key_sub, run_if, kout_alt, vout_alt,
      use_alt);
}

cudaError_t prepare_sort() {
  const int kv8 = (int)(2 * 512 * 8 * sizeof(uint32_t)), kv4 = (int)(2 * 512 * 4 * sizeof(uint32_t));
  cudaError_t e = cudaFuncSetAttribute(k_sort_pass<512, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kv8);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sort_pass<512, 8, 9>, cudaFuncAttributeMaxDynamicSharedMemorySize, kv8);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sort_pass<512, 4, 9>, cudaFuncAttributeMaxDynamicSharedMemorySize, kv4);
  return e;
}

// The record sort by depth (the frame's depth keys: float bits of the
// ordering depth, INVALID_KEY for records that cover no tile).  Every valid
// depth exceeds the nearest near plane, so key - bits(near) keeps the order
// and, for depths below 2^16 x near (13 km at 0.2 m), fits in 27 bits:
// three passes of 9-bit digits, the first over every record (dropping the
// invalid ones), the next two over the valid ones.  A frame with a larger
// key (fd->depth_wide, set by the projection) takes a fourth pass on bits
// 24-31 (it overlaps the third digit, which LSD order allows: the pass is
// stable).  Buffers: (k0, v0), (k1, v1) ping-pong, (k2, v2) the result in
// either case (the third pass writes (k2, v2), or (k0, v0) when the fourth
// follows).  hist: the projection's histograms, 3 x 512 (9-bit digits)
// then 256 (bits 24-31), of the valid keys minus the base.
void launch_depth_sort(const uint32_t* kin, uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, uint32_t* k2,
                       uint32_t* v2, const uint32_t* n_in, const uint32_t* n_valid, int slot_base, FrameDev* fd,
                       SortBufs sb, const uint32_t* hist, int n_sm, cudaStream_t s) {
  sort_pass<512, 8, 9>(n_sm * 2, s, kin, nullptr, k0, v0, n_in, 0, hist, 1, sb.status, fd, slot_base,
                       &fd->depth_base);
  sort_pass<512, 4, 9>(n_sm * 2, s, k0, v0, k1, v1, n_valid, 9, hist + 512, 0, sb.status, fd, slot_base + 1);
  sort_pass<512, 4, 9>(n_sm * 2, s, k1, v1, k2, v2, n_valid, 18, hist + 1024, 0, sb.status, fd, slot_base + 2,
                       nullptr, nullptr, k0, v0, &fd->depth_wide);
  sort_pass<512, 4, 8>(n_sm * 2, s, k0, v0, k2, v2, n_valid, 24, hist + 1536, 0, sb.status, fd, slot_base + 3,
                       nullptr, &fd->depth_wide);
}

// Sort n_in (from device memory) pairs on bits [0, bits).  drop_invalid:
// keys equal to INVALID_KEY are removed (their count is not part of the
// output; *n_valid_out receives the kept count).  Ping-pongs between
// (k0, v0) and (k1, v1); *kout / *vout get the buffers holding the result.
// Uses counter / epoch slots slot_base .. slot_base + passes - 1.  ipt 8
// (the record sort: its first pass runs over every record, invalid ones
// included, in 4096-key tiles; the later passes over the valid ones in
// 2048-key tiles) or 16 (4096-key tiles throughout).
void launch_sort_impl(const uint32_t* kin, const uint32_t* vin, uint32_t* k0, uint32_t* v0, uint32_t* k1,
                      uint32_t* v1, const uint32_t* n_in, uint32_t* n_valid_out, int bits, int drop_invalid,
                      int slot_base, FrameDev* fd, SortBufs sb, int n_sm, cudaStream_t s, uint32_t** kout,
                      uint32_t** vout, int ipt, const uint32_t* hist) {
  const int npass = (bits + 7) / 8;
  if (!hist) {
    cudaMemsetAsync(sb.hist, 0, sizeof(uint32_t) * 4 * 256, s);
    k_sort_hist<<<n_sm * 4, 256, 0, s>>>(kin, n_in, npass, drop_invalid, sb.hist, n_valid_out);
    hist = sb.hist;
  }
  const uint32_t* ci = kin;
  const uint32_t* cv = vin;
  for (int p = 0; p < npass; ++p) {
    uint32_t* ok = (p % 2 == 0) ? k0 : k1;
    uint32_t* ov = (p % 2 == 0) ? v0 : v1;
    const uint32_t* np = (p == 0 || !drop_invalid) ? n_in : n_valid_out;
    if (ipt == 8 && p > 0)
      sort_pass<512, 4>(n_sm * 2, s, ci, cv, ok, ov, np, 8 * p, hist + p * 256, 0, sb.status, fd, slot_base + p);
    else
      sort_pass<512, 8>(n_sm * 2, s, ci, cv, ok, ov, np, 8 * p, hist + p * 256, p == 0 ? drop_invalid : 0, sb.status, fd,
                        slot_base + p);
    ci = ok;
    cv = ov;
  }
  *kout = const_cast<uint32_t*>(ci);
  *vout = const_cast<uint32_t*>(cv);
}

}  // namespace gsc
