// Cache-centric reuse of derived Gaussians (K2; Sec. 4, Alg. 1, Eq. 4).
//
// One cache per derivation view: a pool of S lines, each holding the derived
// attributes of one anchor's k Gaussians in float16 (24 bytes per Gaussian),
// the anchor id and the frame it was decoded in, plus a per-anchor line
// index ("anchor indices are translated to the cache indices by index
// mapping").  Per frame, all on the device:
//   tick     t += 1
//   probe    per visible anchor: hit (valid line with age <= depth), refresh
//            (valid line, older than depth) or new (no valid line; lines past
//            D_max are invalid); misses go to a work list for the decoder;
//            per line: free iff unused or past D_max
//   scans    ranks of new anchors (ascending) and of free lines (ascending)
//   assign   the i-th new anchor takes the i-th free line (none left: decoded
//            but not cached); decoded lines are stamped with t
//   policy   next depth = round(D_max (1 - misses / visible)) in [1, D_max]
//            (Eq. 4, linear guiding function), computed in integers.
// The decoder writes fresh attributes of misses into their lines; the
// projection reads hits from their lines.
#include "gsc_internal.cuh"

namespace gsc {

__global__ void k_cache_tick(CacheDev* caches, int n) {
  const int c = threadIdx.x;
  if (c >= n || !caches[c].active) return;
  uint32_t* st = caches[c].state;
  st[CS_T] += 1u;
  st[CS_MISSES] = 0;
  st[CS_NEW] = 0;
  st[CS_FREE] = 0;
}

__global__ void k_cache_probe(CacheDev* __restrict__ caches, int c, const FrameDev* __restrict__ fd,
                              uint32_t* const* __restrict__ vis) {
  const CacheDev cd = caches[c];
  const uint32_t V = fd->vis_count[c];
  const uint32_t t = cd.state[CS_T], depth = cd.state[CS_DEPTH], D = cd.state[CS_DMAX];
  const uint32_t* ids = vis[c];
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t vi = blockIdx.x * blockDim.x + threadIdx.x; vi < V; vi += stride) {
    const uint32_t a = ids[vi];
    const uint32_t s = cd.slot_of[a];
    bool valid = s < cd.S && cd.slot_anchor[s] == a;
    const uint32_t age = valid ? t - cd.slot_frame[s] : 0xFFFFFFFFu;
    valid = valid && age <= D;
    const bool hit = valid && age <= depth;
    cd.vstat[vi] = hit ? (s | LINE_HIT) : (valid ? s : LINE_NONE);
    cd.new_flag[vi] = valid ? 0u : 1u;
    if (!hit) cd.miss[atomicAdd(&cd.state[CS_MISSES], 1u)] = vi;
  }
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < cd.S; s += stride)
    cd.free_flag[s] = (cd.slot_anchor[s] == 0xFFFFFFFFu || t - cd.slot_frame[s] > D) ? 1u : 0u;
}

__global__ void k_cache_free_list(CacheDev* __restrict__ caches, int c) {
  const CacheDev cd = caches[c];
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < cd.S; s += gridDim.x * blockDim.x)
    if (cd.free_flag[s]) cd.free_list[cd.free_rank[s]] = s;
}

__global__ void k_cache_assign(CacheDev* __restrict__ caches, int c, const FrameDev* __restrict__ fd,
                               uint32_t* const* __restrict__ vis) {
  const CacheDev cd = caches[c];
  const uint32_t V = fd->vis_count[c];
  const uint32_t t = cd.state[CS_T], n_free = cd.state[CS_FREE];
  const uint32_t* ids = vis[c];
  for (uint32_t vi = blockIdx.x * blockDim.x + threadIdx.x; vi < V; vi += gridDim.x * blockDim.x) {
    const uint32_t st = cd.vstat[vi];
    if (st & LINE_HIT) continue;
    const uint32_t a = ids[vi];
    uint32_t line = st;
    if (cd.new_flag[vi]) {
      const uint32_t rank = cd.new_rank[vi];
      line = rank < n_free ? cd.free_list[rank] : LINE_NONE;
      cd.vstat[vi] = line;
    }
    if (line == LINE_NONE) continue;
    cd.slot_anchor[line] = a;
    cd.slot_frame[line] = t;
    cd.slot_of[a] = line;
  }
}

// replay != 0: the frame's decisions and the depth update were already made
// by an earlier attempt at the same frame; only the frame counts are restated.
__global__ void k_cache_policy(CacheDev* caches, int n, FrameDev* fd, int replay) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint32_t hits = 0;
  for (int c = 0; c < n; ++c) {
    if (!caches[c].active) continue;
    uint32_t* st = caches[c].state;
    const uint32_t V = fd->vis_count[c], m = st[CS_MISSES], D = st[CS_DMAX];
    st[CS_VIS] = V;
    hits += V - m;
    if (!replay && V > 0) {
      const unsigned long long num = 2ull * D * (V - m) + V;
      uint32_t d = (uint32_t)(num / (2ull * V));
      st[CS_DEPTH] = d < 1u ? 1u : (d > D ? D : d);
    }
    if (c == 0) fd->cache_depth = st[CS_DEPTH];
  }
  fd->n_derived = fd->n_items - hits;
}

// caches: device array; host: its host-side mirror (same device pointers).
void launch_cache_frame(CacheDev* caches, const CacheDev* host, int n_caches, FrameDev* fd, uint32_t* const* vis,
                        unsigned long long* scan_status, int n_sm, cudaStream_t s) {
  k_cache_tick<<<1, 32, 0, s>>>(caches, n_caches);
  for (int c = 0; c < n_caches; ++c) {
    if (!host[c].active) continue;
    const CacheDev& h = host[c];
    k_cache_probe<<<n_sm * 4, 256, 0, s>>>(caches, c, fd, vis);
    launch_scan_u32(h.new_flag, nullptr, &fd->vis_count[c], h.new_rank, h.state + CS_NEW, scan_status, fd,
                    SLOT_CACHE + 2 * c, n_sm, s);
    launch_scan_u32(h.free_flag, nullptr, h.state + CS_S, h.free_rank, h.state + CS_FREE, scan_status, fd,
                    SLOT_CACHE + 2 * c + 1, n_sm, s);
    k_cache_free_list<<<n_sm * 4, 256, 0, s>>>(caches, c);
    k_cache_assign<<<n_sm * 4, 256, 0, s>>>(caches, c, fd, vis);
  }
}

void launch_cache_policy(CacheDev* caches, int n_caches, FrameDev* fd, bool replay, cudaStream_t s) {
  k_cache_policy<<<1, 32, 0, s>>>(caches, n_caches, fd, replay ? 1 : 0);
}

}  // namespace gsc
