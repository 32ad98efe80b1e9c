// Derivation (K3f/K4) fused with projection (K5), float32 on CUDA cores.
//
// Per visible anchor of a derivation view (Eq. 3):
//   d = (x_a - p)/|x_a - p|, x = [f_a ; d],
//   h_h = ReLU(W1_h^T x + b1_h) for the opacity, colour and covariance heads,
//   z_h = W2_h^T h_h + b2_h,
// followed per Gaussian by the activations, the mask, the per-Gaussian
// broadcast of the anchor's scale and position (the paper's "combine"
// operators, Sec. 6) and the EWA projection + exact tile count for every
// camera the view feeds (Eq. 1-2, Sec. 6).  Derived attributes never go to
// HBM; only projected records do.
//
// A block takes tiles of 64 visible anchors:
//   phase 0  gather features (coalesced 128-byte rows) and view directions
//            into shared memory, transposed: X^T [36][64]
//   phase 1  H = ReLU(X W1cat + b1) [64 x 96]: each thread a 4 x 12 register
//            block (48 accumulators, 4 shared loads per 48 FMAs)
//   phase 2  Z = H W2 + b2 [64 x 110] (block diagonal by head): each thread
//            one anchor, 55 outputs, its hidden row in registers
//   phase 3  640 (anchor, Gaussian) items: activations + projection; records
//            of consecutive items are consecutive, so writes coalesce.
#include "derive_common.cuh"

namespace gsc {

constexpr int DF_NT = 128;
constexpr int DF_TA = 64;            // anchors per tile
constexpr int DF_XS = 64;            // X^T row stride (anchors)
constexpr int DF_HS = 100;           // H row stride (floats): 16-byte aligned, conflict-free float4 rows
constexpr int DF_ZS = 113;           // Z row stride
constexpr int DF_W = (W_FLOATS + 3) / 4 * 4;
constexpr int DF_XZ = (DF_TA * DF_ZS > 36 * DF_XS) ? DF_TA * DF_ZS : 36 * DF_XS;
constexpr int DF_SMEM_FLOATS = DF_W + DF_TA * DF_HS + DF_XZ;
constexpr size_t DF_SMEM_BYTES = (size_t)DF_SMEM_FLOATS * 4;

struct DFMeta {
  uint32_t anchor[DF_TA];
  uint32_t vi[DF_TA];     // visible index within its view
  int ld[DF_TA];          // view slot in the DViewSet (-1: empty item)
  float pos[DF_TA][3];
  float sa[DF_TA];
  uint32_t line[DF_TA];   // cache line the decode rewrites, or LINE_NONE
};

template <int HEAD, int O0, int O1>
__device__ __forceinline__ void df_dots(const float (&h)[NH], const float* __restrict__ s_w, float* zrow) {
#pragma unroll 1
  for (int o = O0; o < O1; o += 5) {
    float acc[5];
#pragma unroll
    for (int u = 0; u < 5; ++u) acc[u] = s_w[WOFF_B2 + o + u];
#pragma unroll
    for (int c4 = 0; c4 < HID / 4; ++c4) {
#pragma unroll
      for (int u = 0; u < 5; ++u) {
        const float4 w = reinterpret_cast<const float4*>(s_w + WOFF_W2T + (o + u) * HID)[c4];
        acc[u] = fmaf(h[HEAD * HID + 4 * c4 + 0], w.x, acc[u]);
        acc[u] = fmaf(h[HEAD * HID + 4 * c4 + 1], w.y, acc[u]);
        acc[u] = fmaf(h[HEAD * HID + 4 * c4 + 2], w.z, acc[u]);
        acc[u] = fmaf(h[HEAD * HID + 4 * c4 + 3], w.w, acc[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < 5; ++u) zrow[o + u] = acc[u];
  }
}

__global__ void __launch_bounds__(DF_NT, 2) k_derive_f32(const ModelDev* __restrict__ models, int model,
                                                         FrameDev* __restrict__ fd, uint32_t* const* __restrict__ vis,
                                                         float4* __restrict__ attrs, float* const* __restrict__ dbg_attrs,
                                                         const CacheDev* __restrict__ caches,
                                                         const DViewSet* __restrict__ tabs) {
  extern __shared__ __align__(16) float s_dyn[];
  float* s_w = s_dyn;
  float* s_h = s_dyn + DF_W;
  float* s_xz = s_h + DF_TA * DF_HS;  // X^T in phases 0-1, Z in phases 2-3
  __shared__ DViewSet S;
  __shared__ DFMeta M;

  const ModelDev md = models[model];
  load_dview_set(S, tabs, fd, model, caches);
  const int nd = S.nd;
  const uint32_t total = S.base[nd];
  const uint32_t ntiles = (total + DF_TA - 1) / DF_TA;
  if (blockIdx.x >= ntiles) return;  // no tile for this block: skip the weight staging
  {
    const float4* src = reinterpret_cast<const float4*>(md.w32);
    for (int i = threadIdx.x; i < W_FLOATS / 4; i += DF_NT) reinterpret_cast<float4*>(s_w)[i] = src[i];
    for (int i = (W_FLOATS / 4) * 4 + threadIdx.x; i < W_FLOATS; i += DF_NT) s_w[i] = md.w32[i];
  }
  __syncthreads();
  const uint32_t rec_cap = fd->n_records;
  const int t = threadIdx.x;

  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // ---- phase 0: item metadata, features and view directions
    if (t < DF_TA) {
      const uint32_t item = tile * DF_TA + t;
      int ld = -1;
      if (item < total) {
        ld = 0;
        while (item >= S.base[ld + 1]) ++ld;
        const uint32_t u = item - S.base[ld];
        const uint32_t vi = S.miss[ld] ? S.miss[ld][u] : u;
        const uint32_t a = vis[S.d[ld]][vi];
        M.anchor[t] = a;
        M.vi[t] = vi;
        uint32_t line = LINE_NONE;
        if (S.vstat[ld]) {
          const uint32_t st = S.vstat[ld][vi];
          if (st != LINE_NONE && !(st & LINE_HIT)) line = st;
        }
        M.line[t] = line;
        const float xa = __ldg(md.px + a), ya = __ldg(md.py + a), za = __ldg(md.pz + a);
        M.pos[t][0] = xa; M.pos[t][1] = ya; M.pos[t][2] = za;
        M.sa[t] = __ldg(md.scale + a);
        float vx = (xa - S.pc[ld][0]) - S.pc[ld][3];
        float vy = (ya - S.pc[ld][1]) - S.pc[ld][4];
        float vz = (za - S.pc[ld][2]) - S.pc[ld][5];
        const float vn = 1.0f / sqrtf(vx * vx + vy * vy + vz * vz);
        s_xz[32 * DF_XS + t] = vx * vn;
        s_xz[33 * DF_XS + t] = vy * vn;
        s_xz[34 * DF_XS + t] = vz * vn;
      } else {
        s_xz[32 * DF_XS + t] = 0.f;
        s_xz[33 * DF_XS + t] = 0.f;
        s_xz[34 * DF_XS + t] = 0.f;
      }
      s_xz[35 * DF_XS + t] = 0.f;
      M.ld[t] = ld;
    }
    __syncthreads();
    for (int u = t; u < DF_TA * (FDIM / 4); u += DF_NT) {
      const int a = u >> 3, part = u & 7;
      float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
      if (M.ld[a] >= 0) f = __ldg(md.feat + (size_t)M.anchor[a] * (FDIM / 4) + part);
      s_xz[(4 * part + 0) * DF_XS + a] = f.x;
      s_xz[(4 * part + 1) * DF_XS + a] = f.y;
      s_xz[(4 * part + 2) * DF_XS + a] = f.z;
      s_xz[(4 * part + 3) * DF_XS + a] = f.w;
    }
    __syncthreads();
    // ---- phase 1: H = ReLU(X W1cat + b1), 4 anchors x 12 hidden per thread
    {
      const int ag = t & 15, hg = t >> 4;
      float acc[4][12];
#pragma unroll
      for (int o = 0; o < 12; ++o) {
        const float b = s_w[WOFF_B1 + 12 * hg + o];
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r][o] = b;
      }
#pragma unroll 5
      for (int k = 0; k < IN; ++k) {
        const float4 x4 = reinterpret_cast<const float4*>(s_xz + k * DF_XS)[ag];
        const float4* wr = reinterpret_cast<const float4*>(s_w + WOFF_W1 + k * NH + 12 * hg);
        const float4 w0 = wr[0], w1 = wr[1], w2 = wr[2];
        const float wv[12] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w, w2.x, w2.y, w2.z, w2.w};
        const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int o = 0; o < 12; ++o) acc[r][o] = fmaf(xv[r], wv[o], acc[r][o]);
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        float4* hp = reinterpret_cast<float4*>(s_h + (4 * ag + r) * DF_HS + 12 * hg);
        hp[0] = make_float4(fmaxf(acc[r][0], 0.f), fmaxf(acc[r][1], 0.f), fmaxf(acc[r][2], 0.f), fmaxf(acc[r][3], 0.f));
        hp[1] = make_float4(fmaxf(acc[r][4], 0.f), fmaxf(acc[r][5], 0.f), fmaxf(acc[r][6], 0.f), fmaxf(acc[r][7], 0.f));
        hp[2] = make_float4(fmaxf(acc[r][8], 0.f), fmaxf(acc[r][9], 0.f), fmaxf(acc[r][10], 0.f), fmaxf(acc[r][11], 0.f));
      }
    }
    __syncthreads();
    // ---- phase 2: Z = H W2 + b2 (block diagonal), one anchor x 55 outputs per thread
    {
      const int a = t & (DF_TA - 1), half = t >> 6;
      float h[NH];
      const float4* hr = reinterpret_cast<const float4*>(s_h + a * DF_HS);
#pragma unroll
      for (int c4 = 0; c4 < NH / 4; ++c4) {
        const float4 v = hr[c4];
        h[4 * c4 + 0] = v.x; h[4 * c4 + 1] = v.y; h[4 * c4 + 2] = v.z; h[4 * c4 + 3] = v.w;
      }
      float* zrow = s_xz + a * DF_ZS;
      if (half == 0) {
        df_dots<0, 0, K>(h, s_w, zrow);
        df_dots<1, K, 4 * K>(h, s_w, zrow);
        df_dots<2, 4 * K, 55>(h, s_w, zrow);
      } else {
        df_dots<2, 55, NOUT>(h, s_w, zrow);
      }
    }
    __syncthreads();
    // ---- phase 3: per (anchor, Gaussian) activations + projection
#pragma unroll 1
    for (int it = t; it < DF_TA * K; it += DF_NT) {
      const int a = it / K, j = it - a * K;
      const int ld = M.ld[a];
      if (ld < 0) continue;
      const float* zr = s_xz + a * DF_ZS;
      float z[11];
      z[0] = zr[j];
#pragma unroll
      for (int u = 0; u < 3; ++u) z[1 + u] = zr[K + 3 * j + u];
#pragma unroll
      for (int u = 0; u < 7; ++u) z[4 + u] = zr[4 * K + 7 * j + u];
      float* dbg = dbg_attrs ? dbg_attrs[S.d[ld]] : nullptr;
      const size_t idx = (size_t)(S.gbase[ld] + M.vi[a]) * K + j;
      uint2* line = M.line[a] != LINE_NONE ? S.lattr[ld] + ((size_t)M.line[a] * K + j) * 3 : nullptr;
      if (idx < rec_cap) gaussian_activate_store(z, j, M.vi[a], M.sa[a], attrs, idx, dbg, line);
    }
    __syncthreads();
  }
}

cudaError_t prepare_derive_f32() {
  return cudaFuncSetAttribute(k_derive_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DF_SMEM_BYTES);
}

void launch_derive_f32(const ModelDev* models, int model, FrameDev* fd, uint32_t* const* vis, float4* attrs,
                       float* const* dbg_attrs, const CacheDev* caches, const DViewSet* tabs, int n_sm,
                       cudaStream_t s) {
  k_derive_f32<<<n_sm * 2, DF_NT, DF_SMEM_BYTES, s>>>(models, model, fd, vis, attrs, dbg_attrs, caches, tabs);
}

}  // namespace gsc
