// Derivation as a sequence of separate operators (the "w/o kernels" row of
// the paper's ablation, Tables 5-6, Sec. 6: a decoder built from generic
// operators, each reading its inputs from and writing its result to device
// memory).  Same arithmetic as the fused float32 kernel (Eq. 3), one launch
// per operator:
//   input     X [n][36]  = [feature (32), unit view direction (3), 0]   (gather)
//   linear1   H [n][96]  = X W1cat + b1                                  (GEMM)
//   relu      H          = max(H, 0)                                    (elementwise)
//   linear2   Z [n][110] = H W2 + b2, block diagonal by head             (GEMM)
//   split     Z -> per-Gaussian streams: opacity [n k], colour [n k][3],
//             covariance [n k][7]                                         (reshape / split)
//   activate  per (anchor, Gaussian): tanh / sigmoid / normalise, the
//             anchor's scale broadcast to its Gaussians, the attributes
//             (and cache line) of the fused kernels                      (combine)
// n counts the decoded anchors of the model's derivation views, in the
// fused kernels' item order.
#include "derive_common.cuh"

namespace gsc {

namespace {
constexpr int UF_NT = 256;
constexpr int UF_XW = 36;  // X row width

__device__ __forceinline__ uint32_t uf_items(const DViewSet* __restrict__ tab) { return tab->base[tab->nd]; }

// item -> (view slot, visible index, anchor) through the decoder's view set
__device__ __forceinline__ int uf_item(const DViewSet& S, uint32_t* const* __restrict__ vis, uint32_t item,
                                       uint32_t& vi, uint32_t& a) {
  int ld = 0;
  while (item >= S.base[ld + 1]) ++ld;
  const uint32_t u = item - S.base[ld];
  vi = S.miss[ld] ? S.miss[ld][u] : u;
  a = vis[S.d[ld]][vi];
  return ld;
}

__global__ void __launch_bounds__(UF_NT) k_op_input(const ModelDev* __restrict__ models, int model,
                                                    uint32_t* const* __restrict__ vis,
                                                    const DViewSet* __restrict__ tabs, float* __restrict__ X) {
  __shared__ DViewSet S;
  stage_table(S, tabs + model);
  __syncthreads();
  const ModelDev& md = models[model];
  const uint32_t n = S.base[S.nd];
  for (uint32_t e = blockIdx.x * UF_NT + threadIdx.x; e < n * UF_XW; e += gridDim.x * UF_NT) {
    const uint32_t item = e / UF_XW, c = e - item * UF_XW;
    uint32_t vi, a;
    const int ld = uf_item(S, vis, item, vi, a);
    float v = 0.f;
    if (c < (uint32_t)FDIM) {
      v = reinterpret_cast<const float*>(md.feat)[(size_t)a * FDIM + c];
    } else if (c < (uint32_t)IN) {
      const float xa = __ldg(md.px + a), ya = __ldg(md.py + a), za = __ldg(md.pz + a);
      const float vx = (xa - S.pc[ld][0]) - S.pc[ld][3];
      const float vy = (ya - S.pc[ld][1]) - S.pc[ld][4];
      const float vz = (za - S.pc[ld][2]) - S.pc[ld][5];
      const float vn = 1.0f / sqrtf(vx * vx + vy * vy + vz * vz);
      v = (c == FDIM ? vx : c == FDIM + 1 ? vy : vz) * vn;
    }
    X[e] = v;
  }
}

// C [n][N] = A [n][KD] B [KD][N] (+ bias): 16 x 16 output tiles, 16-deep
// K slices staged in shared memory.  B is row-major [KD][N] (ldb = N).
template <int KD, int N>
__global__ void __launch_bounds__(256) k_op_gemm(const float* __restrict__ A, int lda, const float* __restrict__ B,
                                                 const float* __restrict__ bias, float* __restrict__ C,
                                                 const DViewSet* __restrict__ tab) {
  __shared__ float sa[16][17], sb[16][17];
  const uint32_t n = uf_items(tab);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int ntn = (N + 15) / 16;
  const uint32_t ntiles = ((n + 15) / 16) * (uint32_t)ntn;
  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint32_t r0 = (tile / ntn) * 16, c0 = (tile % ntn) * 16;
    const uint32_t row = r0 + ty, col = c0 + tx;
    float acc = 0.f;
    for (int k0 = 0; k0 < KD; k0 += 16) {
      sa[ty][tx] = (r0 + ty < n && k0 + tx < KD) ? A[(size_t)(r0 + ty) * lda + k0 + tx] : 0.f;
      sb[ty][tx] = (k0 + ty < KD && c0 + tx < (uint32_t)N) ? B[(size_t)(k0 + ty) * N + c0 + tx] : 0.f;
      __syncthreads();
#pragma unroll
      for (int k = 0; k < 16; ++k) acc = fmaf(sa[ty][k], sb[k][tx], acc);
      __syncthreads();
    }
    if (row < n && col < (uint32_t)N) C[(size_t)row * N + col] = acc + bias[col];
  }
}

__global__ void __launch_bounds__(UF_NT) k_op_relu(float* __restrict__ H, const DViewSet* __restrict__ tab) {
  const uint32_t n = uf_items(tab) * (uint32_t)NH;
  for (uint32_t e = blockIdx.x * UF_NT + threadIdx.x; e < n; e += gridDim.x * UF_NT) H[e] = fmaxf(H[e], 0.f);
}

// Z [n][110] = block-diagonal H W2 + b2: output o belongs to head 0 (o < k),
// 1 (o < 4k) or 2 and reads that head's 32 hidden values; W2T is [110][32].
__global__ void __launch_bounds__(UF_NT) k_op_linear2(const float* __restrict__ H, const float* __restrict__ w32,
                                                      float* __restrict__ Z, const DViewSet* __restrict__ tab) {
  const uint32_t n = uf_items(tab) * (uint32_t)NOUT;
  for (uint32_t e = blockIdx.x * UF_NT + threadIdx.x; e < n; e += gridDim.x * UF_NT) {
    const uint32_t item = e / NOUT, o = e - item * NOUT;
    const int head = o < (uint32_t)K ? 0 : (o < 4u * K ? 1 : 2);
    const float* h = H + (size_t)item * NH + head * HID;
    const float* w = w32 + WOFF_W2T + (size_t)o * HID;
    float acc = w32[WOFF_B2 + o];
#pragma unroll 8
    for (int c = 0; c < HID; ++c) acc = fmaf(h[c], w[c], acc);
    Z[e] = acc;
  }
}

// The head outputs of each anchor regrouped per Gaussian: opacity [n k],
// colour [n k][3], covariance [n k][7].
__global__ void __launch_bounds__(UF_NT) k_op_split(const float* __restrict__ Z, float* __restrict__ op,
                                                    float* __restrict__ col, float* __restrict__ cov,
                                                    const DViewSet* __restrict__ tab) {
  const uint32_t n = uf_items(tab) * (uint32_t)NOUT;
  for (uint32_t e = blockIdx.x * UF_NT + threadIdx.x; e < n; e += gridDim.x * UF_NT) {
    const uint32_t item = e / NOUT, o = e - item * NOUT;
    const float v = Z[e];
    if (o < (uint32_t)K) op[(size_t)item * K + o] = v;
    else if (o < 4u * K) col[(size_t)item * 3 * K + (o - K)] = v;
    else cov[(size_t)item * 7 * K + (o - 4 * K)] = v;
  }
}

__global__ void __launch_bounds__(UF_NT) k_op_activate(const ModelDev* __restrict__ models, int model,
                                                       FrameDev* __restrict__ fd, uint32_t* const* __restrict__ vis,
                                                       const DViewSet* __restrict__ tabs, const float* __restrict__ op,
                                                       const float* __restrict__ col, const float* __restrict__ cov,
                                                       float4* __restrict__ attrs, float* const* __restrict__ dbg_attrs) {
  __shared__ DViewSet S;
  stage_table(S, tabs + model);
  __syncthreads();
  const ModelDev& md = models[model];
  const uint32_t n = S.base[S.nd] * (uint32_t)K;
  const uint32_t rec_cap = fd->n_records;
  for (uint32_t e = blockIdx.x * UF_NT + threadIdx.x; e < n; e += gridDim.x * UF_NT) {
    const uint32_t item = e / K;
    const int j = (int)(e - item * K);
    uint32_t vi, a;
    const int ld = uf_item(S, vis, item, vi, a);
    float z[11];
    z[0] = op[e];
#pragma unroll
    for (int u = 0; u < 3; ++u) z[1 + u] = col[(size_t)e * 3 + u];
#pragma unroll
    for (int u = 0; u < 7; ++u) z[4 + u] = cov[(size_t)e * 7 + u];
    float* dbg = dbg_attrs ? dbg_attrs[S.d[ld]] : nullptr;
    const size_t idx = (size_t)(S.gbase[ld] + vi) * K + j;
    uint2* line = nullptr;
    if (S.vstat[ld]) {
      const uint32_t st = S.vstat[ld][vi];
      if (st != LINE_NONE && !(st & LINE_HIT)) line = S.lattr[ld] + ((size_t)st * K + j) * 3;
    }
    if (idx < rec_cap) gaussian_activate_store(z, j, vi, __ldg(md.scale + a), attrs, idx, dbg, line);
  }
}
}  // namespace

size_t unfused_scratch_floats(size_t items) { return items * (UF_XW + NH + 2 * NOUT); }

void launch_derive_unfused(const ModelDev* models, const ModelDev* h_model, int model, FrameDev* fd,
                           uint32_t* const* vis, float4* attrs, float* const* dbg_attrs, const DViewSet* tabs,
                           float* scratch, size_t items_cap, int n_sm, cudaStream_t s) {
  float* X = scratch;
  float* H = X + items_cap * UF_XW;
  float* Z = H + items_cap * NH;
  float* op = Z + items_cap * NOUT;
  float* col = op + items_cap * K;
  float* cov = col + items_cap * 3 * K;
  const DViewSet* tab = tabs + model;
  const int grid = n_sm * 8;
  k_op_input<<<grid, UF_NT, 0, s>>>(models, model, vis, tabs, X);
  k_op_gemm<IN, NH><<<grid, 256, 0, s>>>(X, UF_XW, h_model->w32 + WOFF_W1, h_model->w32 + WOFF_B1, H, tab);
  k_op_relu<<<grid, UF_NT, 0, s>>>(H, tab);
  k_op_linear2<<<grid, UF_NT, 0, s>>>(H, h_model->w32, Z, tab);
  k_op_split<<<grid, UF_NT, 0, s>>>(Z, op, col, cov, tab);
  k_op_activate<<<grid, UF_NT, 0, s>>>(models, model, fd, vis, tabs, op, col, cov, attrs, dbg_attrs);
}

}  // namespace gsc
