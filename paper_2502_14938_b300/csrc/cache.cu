// Cache-centric reuse of derived Gaussians (K2; Sec. 4, Alg. 1, Eq. 4).
//
// One cache per derivation view: a pool of S lines, each holding the derived
// attributes of one anchor's k Gaussians in float16 (24 bytes per Gaussian),
// the anchor id and the frame it was decoded in, plus a per-anchor line
// index ("anchor indices are translated to the cache indices by index
// mapping").  Per frame, all on the device:
//   tick     t += 1 (in the frame-setup kernel)
//   probe    per visible anchor: hit (valid line with age <= depth), refresh
//            (valid line, older than depth) or new (no valid line; lines past
//            D_max are invalid); misses go to a work list for the decoder;
//            per line below the high-water mark hw: free iff unused or past
//            D_max.  The depth rule runs inside the cull's write pass
//            (cache_probe_depth, as each id is written); k_cache_probe runs
//            the learned rule, and the depth rule when a model of the frame
//            has no anchors (its cull launches nothing)
//   scan     one scan over [free flags of lines 0 .. hw-1 | new flags of the
//            visible anchors]: ranks of those free lines (and their list, in
//            ascending order) and of new anchors (ascending)
//   assign   the i-th new anchor takes the i-th free line (none left: decoded
//            but not cached); decoded lines are stamped with t; then the
//            policy: next depth = H(misses / visible) in [1, D_max] (Eq. 4;
//            H linear, exponential or staged, gsc_depth_guide).
// The free lines in ascending order are those below hw followed by hw,
// hw + 1, ..., S - 1: a line is first used only when every free line below
// it is taken, so no line at or above hw has ever held an anchor.  Scanning
// below hw alone therefore gives the assignment of a scan over all S lines,
// at the cost of the working set (~60k lines on the city path) instead of
// the capacity (400k).
// The decoder writes fresh attributes of misses into their lines; the
// projection reads hits from their lines.
//
// Learned form (reuse = learned): a valid line is reused iff the predictor
// of reuse_common.cuh says so (instead of age <= depth); every decoded line
// is stamped with the unit direction camera -> anchor it was decoded for.
// Collection (training data): between probe and assign, every visible anchor
// holding a valid line gets its predictor inputs and a label comparing the
// line with a fresh derivation of the same frame.
#include "reuse_common.cuh"

namespace gsc {

// Derivation camera of cache c (the unified camera of a stereo pair) and anchor a's position.
__device__ __forceinline__ float anchor_dir(const ModelDev& md, const CamDev& cam, uint32_t a, float d[3]) {
  const float x[3] = {md.px[a], md.py[a], md.pz[a]};
  return pinned_dir(x, cam.pc, cam.pc_lo, d);
}

// rw: predictor weights (learned form), else unused.  The depth-rule form is
// its own instantiation so it does not carry the predictor's registers.
template <bool LEARNED>
__global__ void __launch_bounds__(256) k_cache_probe(CacheDev* __restrict__ caches, int c,
                                                     const FrameDev* __restrict__ fd, uint32_t* const* __restrict__ vis,
                                                     const ModelDev* __restrict__ models,
                                                     const float* __restrict__ rw) {
  __shared__ float s_w[LEARNED ? RPARAM : 1];
  const CacheDev cd = caches[c];
  const uint32_t V = fd->vis_count[c];
  const uint32_t t = cd.state[CS_T], depth = cd.state[CS_DEPTH], D = cd.state[CS_DMAX], hw = cd.state[CS_HW];
  const uint32_t* ids = vis[c];
  const uint32_t stride = gridDim.x * blockDim.x;
  if (LEARNED) {
    for (int i = threadIdx.x; i < RPARAM; i += blockDim.x) s_w[i] = rw[i];
    __syncthreads();
  }
  const CamDev& cam = fd->dcam[c];
  const ModelDev& md = models[cam.model];
  for (uint32_t vi = blockIdx.x * blockDim.x + threadIdx.x; vi < V; vi += stride) {
    const uint32_t a = ids[vi];
    if (!LEARNED) {
      cache_probe_depth(cd, a, vi, t, depth, D, hw, V, const_cast<uint32_t*>(&fd->err));
      continue;
    }
    const uint32_t s = cd.slot_of[a];
    bool valid = s < cd.S && cd.slot_anchor[s] == a;
    const uint32_t age = valid ? t - cd.slot_frame[s] : 0xFFFFFFFFu;
    valid = valid && age <= D;
    bool hit = false;
    if (valid) {
      float dn[3], z[RZ];
      const float dist = anchor_dir(md, cam, a, dn);
      const float4 dl4 = cd.slot_dir[s];
      const float dl[3] = {dl4.x, dl4.y, dl4.z};
      reuse_features(reinterpret_cast<const float*>(md.feat + (size_t)a * (FDIM / 4)), dn, dl, dist, z);
      hit = reuse_logit(s_w, z) >= 0.f;
    }
    cd.vstat[vi] = hit ? (s | LINE_HIT) : (valid ? s : LINE_NONE);
    cd.flags[hw + vi] = valid ? 0u : 1u;
    if (!hit) {
      const uint32_t mi = atomicAdd(&cd.state[CS_MISSES], 1u);
      if (GSC_IN_BOUNDS(mi, V, const_cast<uint32_t*>(&fd->err))) cd.miss[mi] = vi;
    }
  }
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < hw; s += stride) cd.flags[s] = cache_line_free(cd, s, t, D);
  if (blockIdx.x == 0 && threadIdx.x == 0) cd.state[CS_SCAN_N] = hw + V;
}

// Eq. 4 with the guiding function of the configuration (gsc_depth_guide).
__device__ __forceinline__ uint32_t next_depth(uint32_t depth, uint32_t V, uint32_t m, uint32_t D, uint32_t guide) {
  if (V == 0) return depth;
  uint32_t d;
  if (guide == GSC_GUIDE_EXP) {
    const double e = exp((1.0 - (double)m / (double)V) * log((double)D));
    d = (uint32_t)floor(e + 0.5);
  } else if (guide == GSC_GUIDE_STAGED) {
    d = 10ull * m < V ? D : (10ull * m < 3ull * V ? (D + 1u) / 2u : 1u);
  } else {
    const unsigned long long num = 2ull * D * (V - m) + V;
    d = (uint32_t)(num / (2ull * V));
  }
  return d < 1u ? 1u : (d > D ? D : d);
}

__global__ void k_cache_assign(CacheDev* __restrict__ caches, int c, FrameDev* __restrict__ fd,
                               uint32_t* const* __restrict__ vis, const ModelDev* __restrict__ models) {
  const CacheDev cd = caches[c];
  const CamDev& cam = fd->dcam[c];
  const ModelDev& md = models[cam.model];
  const uint32_t V = fd->vis_count[c];
  const uint32_t t = cd.state[CS_T], hw = cd.state[CS_HW];
  // free lines below hw (their flags precede the new flags); then hw .. S-1
  const uint32_t n_free = V ? cd.ranks[hw] : cd.state[CS_SCAN_TOT];
  const uint32_t* ids = vis[c];
  if (blockIdx.x == 0 && threadIdx.x == 0) {  // bookkeeping and the policy for the next frame
    uint32_t* st = cd.state;
    const uint32_t m = st[CS_MISSES];
    const uint32_t n_new = st[CS_SCAN_TOT] - n_free;
    st[CS_VIS] = V;
    st[CS_FREE] = n_free + (cd.S - hw);
    st[CS_NEW] = n_new;
    st[CS_HW_NEXT] = n_new > n_free ? min(cd.S, hw + (n_new - n_free)) : hw;
    st[CS_DEPTH] = next_depth(st[CS_DEPTH], V, m, st[CS_DMAX], st[CS_GUIDE]);
    atomicSub(&fd->n_derived, V - m);
    if (c == 0) fd->cache_depth = st[CS_DEPTH];
  }
  for (uint32_t vi = blockIdx.x * blockDim.x + threadIdx.x; vi < V; vi += gridDim.x * blockDim.x) {
    const uint32_t st = cd.vstat[vi];
    if (st & LINE_HIT) continue;
    const uint32_t a = ids[vi];
    uint32_t line = st;
    if (cd.flags[hw + vi]) {
      const uint32_t rank = cd.ranks[hw + vi] - n_free;
      line = rank < n_free ? cd.free_list[rank] : (rank - n_free < cd.S - hw ? hw + (rank - n_free) : LINE_NONE);
      cd.vstat[vi] = line;
    }
    if (line == LINE_NONE || !GSC_IN_BOUNDS(line, cd.S, &fd->err)) continue;
    cd.slot_anchor[line] = a;
    cd.slot_frame[line] = t;
    cd.slot_of[a] = line;
    float d[3];
    anchor_dir(md, cam, a, d);
    cd.slot_dir[line] = make_float4(d[0], d[1], d[2], 0.f);
  }
}

// Collection: predictor inputs and label of every visible anchor holding a
// valid line, before this frame touches the lines.  Label 1 iff the line and
// the fresh derivation (attrs_fresh, this frame, frame item order) keep the
// same Gaussians and, over the kept ones, |d alpha| <= 1/255 and
// max_channel |d c| * alpha_fresh <= 1/255.
__global__ void k_reuse_label(CacheDev* __restrict__ caches, int c, const FrameDev* __restrict__ fd,
                              uint32_t* const* __restrict__ vis, const ModelDev* __restrict__ models,
                              const float4* __restrict__ attrs_fresh) {
  const CacheDev cd = caches[c];
  const uint32_t V = fd->vis_count[c];
  const uint32_t* ids = vis[c];
  const CamDev& cam = fd->dcam[c];
  const ModelDev& md = models[cam.model];
  const uint32_t item0 = fd->item_base[c];
  const float thr = 1.0f / 255.0f;
  for (uint32_t vi = blockIdx.x * blockDim.x + threadIdx.x; vi < V; vi += gridDim.x * blockDim.x) {
    const uint32_t st = cd.vstat[vi];
    if (st == LINE_NONE) {
      cd.clab[vi] = 255;
      continue;
    }
    const uint32_t s = st & ~LINE_HIT, a = ids[vi];
    float dn[3], z[RZ];
    const float dist = anchor_dir(md, cam, a, dn);
    const float4 dl4 = cd.slot_dir[s];
    const float dl[3] = {dl4.x, dl4.y, dl4.z};
    reuse_features(reinterpret_cast<const float*>(md.feat + (size_t)a * (FDIM / 4)), dn, dl, dist, z);
    float* zo = cd.cz + (size_t)vi * RZ;
#pragma unroll
    for (int k = 0; k < RZ; ++k) zo[k] = z[k];
    bool ok = true;
    for (int j = 0; j < K; ++j) {
      const uint2 h0 = cd.slot_attr[((size_t)s * K + j) * 3];
      const float2 ac = __half22float2(*reinterpret_cast<const __half2*>(&h0.x));
      const float2 cc = __half22float2(*reinterpret_cast<const __half2*>(&h0.y));
      const float4 f = attrs_fresh[3 * ((size_t)(item0 + vi) * K + j)];
      const bool kc = ac.x > 0.f, kf = f.x > 0.f;
      if (kc != kf) ok = false;
      if (kf) {
        const float dc = fmaxf(fmaxf(fabsf(ac.y - f.y), fabsf(cc.x - f.z)), fabsf(cc.y - f.w)) * f.x;
        if (fabsf(ac.x - f.x) > thr || dc > thr) ok = false;
      }
    }
    cd.clab[vi] = ok ? 1 : 0;
  }
}

// A frame rendered again after a buffer grew: its decisions and the depth
// update were made by the first attempt; restate the frame's counts.
__global__ void k_cache_replay_counts(CacheDev* caches, int n, FrameDev* fd) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint32_t hits = 0;
  for (int c = 0; c < n; ++c) {
    if (!caches[c].active) continue;
    const uint32_t* st = caches[c].state;
    hits += fd->vis_count[c] - st[CS_MISSES];
    if (c == 0) fd->cache_depth = st[CS_DEPTH];
  }
  fd->n_derived = fd->n_items - hits;
}

// caches: device array; host: its host-side mirror (same device pointers).
void launch_cache_frame(CacheDev* caches, const CacheDev* host, int n_caches, FrameDev* fd, uint32_t* const* vis,
                        const ModelDev* models, const float* reuse_w, bool learned, const float4* attrs_fresh,
                        unsigned long long* scan_status, int n_sm, cudaStream_t s, bool probed) {
  for (int c = 0; c < n_caches; ++c) {
    if (!host[c].active) continue;
    const CacheDev& h = host[c];
    if (learned)
      k_cache_probe<true><<<n_sm * 4, 256, 0, s>>>(caches, c, fd, vis, models, reuse_w);
    else if (!probed)
      k_cache_probe<false><<<n_sm * 4, 256, 0, s>>>(caches, c, fd, vis, models, reuse_w);
    if (attrs_fresh) k_reuse_label<<<n_sm * 4, 128, 0, s>>>(caches, c, fd, vis, models, attrs_fresh);
    launch_scan_u32(h.flags, nullptr, h.state + CS_SCAN_N, h.ranks, h.state + CS_SCAN_TOT, scan_status, fd,
                    SLOT_CACHE + 2 * c, n_sm, s, h.free_list, h.S, nullptr, nullptr, 0, h.state + CS_HW);
    k_cache_assign<<<n_sm * 4, 256, 0, s>>>(caches, c, fd, vis, models);
  }
}

void launch_cache_replay_counts(CacheDev* caches, int n_caches, FrameDev* fd, cudaStream_t s) {
  k_cache_replay_counts<<<1, 32, 0, s>>>(caches, n_caches, fd);
}

}  // namespace gsc
