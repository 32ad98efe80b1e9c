// Projection (K5): derived attributes -> one record per (camera, Gaussian).
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

__global__ void __launch_bounds__(PJ_NT) k_project(const ModelDev* __restrict__ models, FrameDev* __restrict__ fd,
                                                   uint32_t* const* __restrict__ vis, const float4* __restrict__ attrs,
                                                   const CacheDev* __restrict__ caches, Records rec) {
  __shared__ uint32_t s_ibase[MAXV + 1];
  __shared__ int s_model[MAXV];
  __shared__ const uint32_t* s_vstat[MAXV];
  __shared__ const uint2* s_lattr[MAXV];
  __shared__ ProjCam s_cam[MAXV][2];
  if (threadIdx.x == 0) {
    const int nd = (int)fd->n_dviews;
    for (int d = 0; d < nd; ++d) {
      s_ibase[d] = fd->item_base[d];
      s_model[d] = fd->dcam[d].model;
      const bool cached = caches && d < MAX_CACHES && caches[d].active;
      s_vstat[d] = cached ? caches[d].vstat : nullptr;
      s_lattr[d] = cached ? caches[d].slot_attr : nullptr;
      for (int e = 0; e < 2; ++e) {
        const int ci = fd->dview_cam[d][e];
        ProjCam& pc = s_cam[d][e];
        pc.cam = ci < 0 ? 0xFFFFFFFFu : (uint32_t)ci;
        if (ci < 0) continue;
        const CamDev& c = fd->cam[ci];
        for (int i = 0; i < 9; ++i) pc.R[i] = c.R[i];
        for (int i = 0; i < 3; ++i) {
          pc.t[i] = c.t[i];
          pc.pc[i] = c.pc[i];
          pc.pc_lo[i] = c.pc_lo[i];
          pc.dt[i] = c.dt[i];
        }
        pc.fx = c.fx; pc.fy = c.fy; pc.cx = c.cx; pc.cy = c.cy;
        pc.znear = c.znear; pc.gx = c.gx; pc.gy = c.gy;
        pc.W = c.W; pc.H = c.H;
        pc.rec_base = fd->rec_base[ci];
      }
    }
    s_ibase[nd] = fd->n_items;
  }
  __syncthreads();
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
    const float alpha = a0.x;
    const bool kept = alpha > 0.f;
    const float col[3] = {a0.y, a0.z, a0.w};
    const float s[3] = {a1.x, a1.y, a1.z};
    const float q[4] = {a1.w, a2.x, a2.y, a2.z};
    const float xa = __ldg(md.px + a), ya = __ldg(md.py + a), za = __ldg(md.pz + a);
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
      project_write(pc, rec, r, mu, rel, alpha, kept, col, s, q, TW, TH);
    }
  }
}

void launch_project(const ModelDev* models, FrameDev* fd, uint32_t* const* vis, const float4* attrs,
                    const CacheDev* caches, Records rec, int n_sm, cudaStream_t s) {
  k_project<<<n_sm * 8, PJ_NT, 0, s>>>(models, fd, vis, attrs, caches, rec);
}

}  // namespace gsc
