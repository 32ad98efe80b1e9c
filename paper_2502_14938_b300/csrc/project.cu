// Projection (K5): derived attributes -> one record per (camera, Gaussian).
// With an Octree-GS level fade (beta > 0) a Gaussian's opacity is first
// scaled by min(1, log2(r_a / d) / beta) of its anchor (level >= 1).
//
// One thread per (visible anchor item, Gaussian j) of the whole frame, in
// item order, runs the cheap first test of its records; the records that
// pass are projected across the warp.  Per camera the derivation view
// feeds: EWA projection of the Gaussian (Eq. 1-2), its opacity-aware exact
// tile count (Sec. 6) and the record.  Kept apart from the derivation kernels because this part is
// latency-bound (IEEE divisions and square roots of the coverage test) and
// wants the full occupancy of a small kernel.
#include "derive_common.cuh"

namespace gsc {

constexpr int PJ_NT = 256;
// staging rows of a surviving record's inputs (one column per owning lane)
enum : int { PS_DJ = 0, PS_VI, PS_X, PS_O = PS_X + 3, PS_COL = PS_O + 3, PS_S = PS_COL + 3, PS_Q = PS_S + 3,
             PS_A = PS_Q + 4, PS_WORDS = PS_A + 2 };

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
  __shared__ uint32_t s_h[DEPTH_HIST_WORDS];  // digit histograms of this block's valid depth keys
  __shared__ uint32_t s_nv, s_wide, s_dbase;
  __shared__ uint8_t s_own[PJ_NT / 32][64];  // per warp: owning lane of each surviving record
  __shared__ float s_stage[PJ_NT / 32][PS_WORDS][32];  // per warp: the owners' record inputs
  for (int i = threadIdx.x; i < DEPTH_HIST_WORDS; i += PJ_NT) s_h[i] = 0;
  if (threadIdx.x == 0) {
    s_nv = s_wide = 0;
    s_dbase = fd->depth_base;
  }
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
  const uint32_t lane = threadIdx.x & 31u;
  uint8_t* owners = s_own[threadIdx.x >> 5];
  float (*stage)[32] = s_stage[threadIdx.x >> 5];
  // Warp-uniform grid stride: each lane takes one (item, Gaussian) and runs
  // the record's first test for both cameras; records that fail it are only
  // their invalid key.  The rest (about a third of the records on the city
  // path) are then projected 32 at a time across the warp, their inputs
  // moved from the owning lane by shuffles, so that the EWA projection and
  // the exact tile count run on full warps.
  for (uint32_t gb = blockIdx.x * PJ_NT + (threadIdx.x & ~31u); gb < n; gb += gridDim.x * PJ_NT) {
    const uint32_t g = gb + lane;
    const bool act = g < n && g < rec_cap;
    uint32_t dj = 0, vi = 0, vmask = 0;
    float xa = 0.f, ya = 0.f, za = 0.f, o3[3] = {0.f, 0.f, 0.f}, al[2] = {0.f, 0.f};
    float col[3] = {0.f, 0.f, 0.f}, s[3] = {0.f, 0.f, 0.f}, q[4] = {0.f, 0.f, 0.f, 0.f};
    if (act) {
      const uint32_t item = g / (uint32_t)K;
      const int j = (int)(g - item * (uint32_t)K);
      int d = 0;
      while (item >= s_ibase[d + 1]) ++d;
      vi = item - s_ibase[d];
      dj = (uint32_t)d | ((uint32_t)j << 8);
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
      xa = __ldg(md.px + a); ya = __ldg(md.py + a); za = __ldg(md.pz + a);
      // Octree-GS level fade, from this frame's distance (so after the cache),
      // measured from the camera whose filter selected the anchor: the
      // derivation camera, or in an exact stereo view each eye itself
      const bool fade = md.lod_beta > 0.f && __ldg(md.lod_r + a) < INFINITY;
      const uint8_t eb = s_eyes[d] ? s_eyes[d][vi] : (uint8_t)3;
      float alpha = a0.x;
      if (fade && !s_eyes[d]) alpha *= lod_fade(md, a, xa, ya, za, fd->dcam[d].pc);
      const bool kept = alpha > 0.f;
      col[0] = a0.y; col[1] = a0.z; col[2] = a0.w;
      s[0] = a1.x; s[1] = a1.y; s[2] = a1.z;
      q[0] = a1.w; q[1] = a2.x; q[2] = a2.y; q[3] = a2.z;
      const float* op = md.offs + ((size_t)a * K + j) * 3;
      o3[0] = __ldg(op); o3[1] = __ldg(op + 1); o3[2] = __ldg(op + 2);
      const float mu[3] = {__fadd_rn(xa, o3[0]), __fadd_rn(ya, o3[1]), __fadd_rn(za, o3[2])};
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const ProjCam& pc = s_cam[d][e];
        if (pc.cam == 0xFFFFFFFFu) continue;
        const uint32_t r = pc.rec_base + vi * K + (uint32_t)j;
        if (r >= rec_cap) continue;
        float alpha_e = alpha;
        bool kept_e = kept;
        if (s_eyes[d]) {  // exact stereo view: this eye draws only the anchors its own filter kept
          if (fade) alpha_e = a0.x * lod_fade(md, a, xa, ya, za, pc.pc);
          kept_e = ((eb >> e) & 1u) && alpha_e > 0.f;
        }
        al[e] = alpha_e;
        if (record_may_draw(pc, mu, alpha_e, kept_e))
          vmask |= 1u << e;
        else
          rec.key[r] = INVALID_KEY;
      }
    }
    // the warp's surviving records: camera 0's owners, then camera 1's; each
    // owner leaves its record inputs in the warp's staging rows
    const uint32_t m0 = __ballot_sync(0xffffffffu, vmask & 1u), m1 = __ballot_sync(0xffffffffu, (vmask >> 1) & 1u);
    const uint32_t n0 = __popc(m0), nt = n0 + __popc(m1);
    if (nt == 0) continue;
    const uint32_t below = (1u << lane) - 1u;
    if (vmask & 1u) owners[__popc(m0 & below)] = (uint8_t)lane;
    if (vmask & 2u) owners[n0 + __popc(m1 & below)] = (uint8_t)lane;
    if (vmask) {
      stage[PS_DJ][lane] = __uint_as_float(dj);
      stage[PS_VI][lane] = __uint_as_float(vi);
      stage[PS_X][lane] = xa; stage[PS_X + 1][lane] = ya; stage[PS_X + 2][lane] = za;
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        stage[PS_O + u][lane] = o3[u];
        stage[PS_COL + u][lane] = col[u];
        stage[PS_S + u][lane] = s[u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) stage[PS_Q + u][lane] = q[u];
      stage[PS_A][lane] = al[0]; stage[PS_A + 1][lane] = al[1];
    }
    __syncwarp();
    for (uint32_t k = lane; k < nt; k += 32u) {
      const int src = owners[k];
      const int e = k < n0 ? 0 : 1;
      const uint32_t w_dj = __float_as_uint(stage[PS_DJ][src]), w_vi = __float_as_uint(stage[PS_VI][src]);
      const int d = (int)(w_dj & 0xFFu), j = (int)(w_dj >> 8);
      const ProjCam& pc = s_cam[d][e];
      const uint32_t r = pc.rec_base + w_vi * K + (uint32_t)j;
      const float wx = stage[PS_X][src], wy = stage[PS_X + 1][src], wz = stage[PS_X + 2][src];
      const float wo[3] = {stage[PS_O][src], stage[PS_O + 1][src], stage[PS_O + 2][src]};
      const float mu[3] = {__fadd_rn(wx, wo[0]), __fadd_rn(wy, wo[1]), __fadd_rn(wz, wo[2])};
      const float rel[3] = {((wx - pc.pc[0]) - pc.pc_lo[0]) + wo[0], ((wy - pc.pc[1]) - pc.pc_lo[1]) + wo[1],
                            ((wz - pc.pc[2]) - pc.pc_lo[2]) + wo[2]};
      const float wcol[3] = {stage[PS_COL][src], stage[PS_COL + 1][src], stage[PS_COL + 2][src]};
      const float ws[3] = {stage[PS_S][src], stage[PS_S + 1][src], stage[PS_S + 2][src]};
      const float wq[4] = {stage[PS_Q][src], stage[PS_Q + 1][src], stage[PS_Q + 2][src], stage[PS_Q + 3][src]};
      const uint32_t key = project_write(pc, rec, r, mu, rel, stage[PS_A + e][src], true, wcol, ws, wq, TW, TH);
      if (key != INVALID_KEY) {  // the depth sort's digits of key - base: 3 x 9 bits, and bits 24-31
        const uint32_t kb = key - s_dbase;
        atomicAdd(&s_h[kb & 511u], 1u);
        atomicAdd(&s_h[512 + ((kb >> 9) & 511u)], 1u);
        atomicAdd(&s_h[1024 + ((kb >> 18) & 511u)], 1u);
        atomicAdd(&s_h[1536 + (kb >> 24)], 1u);
        if (kb >> 27) s_wide = 1u;
        atomicAdd(&s_nv, 1u);
      }
    }
    __syncwarp();  // owners and the staging rows are rewritten by the next round
  }
  __syncthreads();
  for (int i = threadIdx.x; i < DEPTH_HIST_WORDS; i += PJ_NT) {
    const uint32_t c = s_h[i];
    if (c) atomicAdd(&fd->hist_depth[i], c);
  }
  if (threadIdx.x == 0 && s_nv) atomicAdd(&fd->n_valid, s_nv);
  if (threadIdx.x == 0 && s_wide) atomicOr(&fd->depth_wide, 1u);
}

void launch_project(const ModelDev* models, FrameDev* fd, uint32_t* const* vis, const float4* attrs,
                    const CacheDev* caches, Records rec, const ProjTab* ptab, int n_sm, cudaStream_t s) {
  // one wave of resident blocks (four per SM) striding over the Gaussians:
  // half the per-block histogram flushes of two waves
  k_project<<<n_sm * 4, PJ_NT, 0, s>>>(models, fd, vis, attrs, caches, rec, ptab);
}

// ------------------------------------------------------------------ frame tables
// One warp after the cache decisions (frame_tables_warp, derive_common.cuh).
__global__ void k_tables(const FrameDev* __restrict__ fd, const CacheDev* __restrict__ caches,
                         uint8_t* const* __restrict__ eyes, DViewSet* __restrict__ tabs, ProjTab* __restrict__ ptab,
                         int n_models) {
  frame_tables_warp(fd, caches, eyes, tabs, ptab, n_models, (int)(threadIdx.x & 31u));
}

size_t dview_set_bytes() { return sizeof(DViewSet); }
size_t proj_tab_bytes() { return sizeof(ProjTab); }

void launch_tables(const FrameDev* fd, const CacheDev* caches, uint8_t* const* eyes, DViewSet* tabs, ProjTab* ptab,
                   int n_models, cudaStream_t s) {
  k_tables<<<1, 32, 0, s>>>(fd, caches, eyes, tabs, ptab, n_models);
}

}  // namespace gsc
