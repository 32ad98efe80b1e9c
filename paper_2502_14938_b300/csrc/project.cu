// Projection (K5): derived attributes -> one record per (camera, Gaussian).
// With an Octree-GS level fade (beta > 0) a Gaussian's opacity is first
// scaled by min(1, log2(r_a / d) / beta) of its anchor (level >= 1).
//
// One thread per (visible anchor item, Gaussian j) of the whole frame, in
// item order, so the records of consecutive threads are consecutive and the
// writes coalesce.  Per camera the derivation view feeds: EWA projection of
// the Gaussian (Eq. 1-2), its opacity-aware exact tile count (Sec. 6) and
// the record.  Kept apart from the derivation kernels because this part is
// latency-bound (IEEE divisions and square roots of the coverage test) and
// wants the full occupancy of a small kernel.
#include "derive_common.cuh"

namespace gsc {

constexpr int PJ_NT = 256;

// Octree-GS level fade of anchor a (level >= 1) seen from centre pc: w =
// clamp(u / beta, 0, 1), u = log2(r_a / d) the levels it lies inside its
// switching distance.  d^2 is the cull's float32 squared distance (same
// operations, same centre), so u >= 0 exactly for every anchor that filter
// kept; u = log1p((r^2 - d^2) / d^2) / (2 ln 2), with r^2 - d^2 rounded once,
// stays accurate relative to itself as the anchor nears its switch.
__device__ __forceinline__ float lod_fade(const ModelDev& md, uint32_t a, float xa, float ya, float za,
                                          const float* pc) {
  const float ra = __ldg(md.lod_r + a);
  const float dx = __fsub_rn(xa, pc[0]), dy = __fsub_rn(ya, pc[1]), dz = __fsub_rn(za, pc[2]);
  const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
  const float u = 0.72134752f * log1pf(__fdiv_rn(fmaf(ra, ra, -d2), d2));
  return fminf(1.f, fmaxf(0.f, __fdiv_rn(u, md.lod_beta)));
}

__global__ void __launch_bounds__(PJ_NT, 4) k_project(const ModelDev* __restrict__ models, FrameDev* __restrict__ fd,
                                                   uint32_t* const* __restrict__ vis, const float4* __restrict__ attrs,
                                                   const CacheDev* __restrict__ caches, Records rec,
                                                   const ProjTab* __restrict__ ptab) {
  __shared__ ProjTab P;
  __shared__ uint32_t s_h[4][256];  // digit histograms of this block's valid depth keys
  __shared__ uint32_t s_nv;
  for (int i = threadIdx.x; i < 4 * 256; i += PJ_NT) (&s_h[0][0])[i] = 0;
  if (threadIdx.x == 0) s_nv = 0;
  if (ptab) {
    stage_table(P, ptab);
  } else if (threadIdx.x == 0) {
    const int nd = (int)fd->n_dviews;
    for (int d = 0; d < nd; ++d) {
      P.ibase[d] = fd->item_base[d];
      P.model[d] = fd->dcam[d].model;
      const bool cached = caches && d < MAX_CACHES && caches[d].active;
      P.vstat[d] = cached ? caches[d].vstat : nullptr;
      P.lattr[d] = cached ? caches[d].slot_attr : nullptr;
      P.eyes[d] = nullptr;  // (frames always pass the table; exact stereo views need it)
      for (int e = 0; e < 2; ++e) fill_projcam(P.cam[d][e], fd, fd->dview_cam[d][e]);
    }
    P.ibase[nd] = fd->n_items;
  }
  __syncthreads();
  const uint32_t* s_ibase = P.ibase;
  const int* s_model = P.model;
  const uint32_t* const* s_vstat = P.vstat;
  const uint2* const* s_lattr = P.lattr;
  const uint8_t* const* s_eyes = P.eyes;
  ProjCam (*s_cam)[2] = P.cam;
  const uint32_t n = fd->n_items * (uint32_t)K;
  const uint32_t rec_cap = fd->n_records;
  const int TW = (int)fd->tile_w, TH = (int)fd->tile_h;
  for (uint32_t g = blockIdx.x * PJ_NT + threadIdx.x; g < n; g += gridDim.x * PJ_NT) {
    if (g >= rec_cap) break;
    const uint32_t item = g / (uint32_t)K;
    const int j = (int)(g - item * (uint32_t)K);
    int d = 0;
    while (item >= s_ibase[d + 1]) ++d;
    const uint32_t vi = item - s_ibase[d];
    const ModelDev& md = models[s_model[d]];
    const uint32_t a = vis[d][vi];
    float4 a0, a1, a2;
    const uint32_t st = s_vstat[d] ? s_vstat[d][vi] : LINE_NONE;
    if (st & LINE_HIT) {  // reuse: the float16 line decoded in an earlier frame
      const uint2* l = s_lattr[d] + ((size_t)(st & ~LINE_HIT) * K + j) * 3;
      const uint2 h0 = l[0], h1 = l[1], h2 = l[2];
      const float2 x0 = __half22float2(*reinterpret_cast<const __half2*>(&h0.x));
      const float2 x1 = __half22float2(*reinterpret_cast<const __half2*>(&h0.y));
      const float2 x2 = __half22float2(*reinterpret_cast<const __half2*>(&h1.x));
      const float2 x3 = __half22float2(*reinterpret_cast<const __half2*>(&h1.y));
      const float2 x4 = __half22float2(*reinterpret_cast<const __half2*>(&h2.x));
      const float2 x5 = __half22float2(*reinterpret_cast<const __half2*>(&h2.y));
      a0 = make_float4(x0.x, x0.y, x1.x, x1.y);
      a1 = make_float4(x2.x, x2.y, x3.x, x3.y);
      a2 = make_float4(x4.x, x4.y, x5.x, x5.y);
    } else {
      a0 = attrs[3 * (size_t)g + 0];
      a1 = attrs[3 * (size_t)g + 1];
      a2 = attrs[3 * (size_t)g + 2];
    }
    const float xa = __ldg(md.px + a), ya = __ldg(md.py + a), za = __ldg(md.pz + a);
    // Octree-GS level fade, from this frame's distance (so after the cache),
    // measured from the camera whose filter selected the anchor: the
    // derivation camera, or in an exact stereo view each eye itself
    const bool fade = md.lod_beta > 0.f && __ldg(md.lod_r + a) < INFINITY;
    const uint8_t eb = s_eyes[d] ? s_eyes[d][vi] : (uint8_t)3;
    float alpha = a0.x;
    if (fade && !s_eyes[d]) alpha *= lod_fade(md, a, xa, ya, za, fd->dcam[d].pc);
    const bool kept = alpha > 0.f;
    const float col[3] = {a0.y, a0.z, a0.w};
    const float s[3] = {a1.x, a1.y, a1.z};
    const float q[4] = {a1.w, a2.x, a2.y, a2.z};
    const float* op = md.offs + ((size_t)a * K + j) * 3;
    const float o3[3] = {__ldg(op), __ldg(op + 1), __ldg(op + 2)};
    const float mu[3] = {__fadd_rn(xa, o3[0]), __fadd_rn(ya, o3[1]), __fadd_rn(za, o3[2])};
#pragma unroll 1
    for (int e = 0; e < 2; ++e) {
      const ProjCam& pc = s_cam[d][e];
      if (pc.cam == 0xFFFFFFFFu) continue;
      const uint32_t r = pc.rec_base + vi * K + (uint32_t)j;
      if (r >= rec_cap) continue;
      const float rel[3] = {((xa - pc.pc[0]) - pc.pc_lo[0]) + o3[0], ((ya - pc.pc[1]) - pc.pc_lo[1]) + o3[1],
                            ((za - pc.pc[2]) - pc.pc_lo[2]) + o3[2]};
      float alpha_e = alpha;
      bool kept_e = kept;
      if (s_eyes[d]) {  // exact stereo view: this eye draws only the anchors its own filter kept
        if (fade) alpha_e = a0.x * lod_fade(md, a, xa, ya, za, pc.pc);
        kept_e = ((eb >> e) & 1u) && alpha_e > 0.f;
      }
      const uint32_t key = project_write(pc, rec, r, mu, rel, alpha_e, kept_e, col, s, q, TW, TH);
      if (key != INVALID_KEY) {
#pragma unroll
        for (int p = 0; p < 4; ++p) atomicAdd(&s_h[p][(key >> (8 * p)) & 0xFFu], 1u);
        atomicAdd(&s_nv, 1u);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * 256; i += PJ_NT) {
    const uint32_t c = (&s_h[0][0])[i];
    if (c) atomicAdd(&fd->hist_depth[i], c);
  }
  if (threadIdx.x == 0 && s_nv) atomicAdd(&fd->n_valid, s_nv);
}

void launch_project(const ModelDev* models, FrameDev* fd, uint32_t* const* vis, const float4* attrs,
                    const CacheDev* caches, Records rec, const ProjTab* ptab, int n_sm, cudaStream_t s) {
  // one wave of resident blocks (four per SM) striding over the Gaussians:
  // half the per-block histogram flushes of two waves
  k_project<<<n_sm * 4, PJ_NT, 0, s>>>(models, fd, vis, attrs, caches, rec, ptab);
}

// ------------------------------------------------------------------ frame tables
// One warp after the cache kernels: lane d fills derivation view d's entries
// of the projection table and of its model's decoder view set (at its rank
// among the model's views); lane m closes model m's set.
__global__ void k_tables(const FrameDev* __restrict__ fd, const CacheDev* __restrict__ caches,
                         uint8_t* const* __restrict__ eyes, DViewSet* __restrict__ tabs, ProjTab* __restrict__ ptab,
                         int n_models) {
  const int lane = (int)(threadIdx.x & 31u);
  const int nd = (int)fd->n_dviews;
  auto work = [&](int d) -> uint32_t {
    const bool cached = caches && d < MAX_CACHES && caches[d].active;
    return cached ? caches[d].state[CS_MISSES] : fd->vis_count[d];
  };
  if (lane < nd) {
    const int d = lane, m = fd->dcam[d].model;
    const bool cached = caches && d < MAX_CACHES && caches[d].active;
    ptab->ibase[d] = fd->item_base[d];
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
    S.gbase[r] = fd->item_base[d];
    S.miss[r] = cached ? caches[d].miss : nullptr;
    S.vstat[r] = cached ? caches[d].vstat : nullptr;
    S.lattr[r] = cached ? caches[d].slot_attr : nullptr;
    for (int u = 0; u < 3; ++u) {
      S.pc[r][u] = fd->dcam[d].pc[u];
      S.pc[r][3 + u] = fd->dcam[d].pc_lo[u];
    }
    for (int e = 0; e < 2; ++e) {
      fill_projcam(ptab->cam[d][e], fd, fd->dview_cam[d][e]);
      fill_projcam(S.cam[r][e], fd, fd->dview_cam[d][e]);
    }
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

size_t dview_set_bytes() { return sizeof(DViewSet); }
size_t proj_tab_bytes() { return sizeof(ProjTab); }

void launch_tables(const FrameDev* fd, const CacheDev* caches, uint8_t* const* eyes, DViewSet* tabs, ProjTab* ptab,
                   int n_models, cudaStream_t s) {
  k_tables<<<1, 32, 0, s>>>(fd, caches, eyes, tabs, ptab, n_models);
}

}  // namespace gsc
