// Derivation on the 5th-generation tensor cores (tcgen05), BF16 inputs with
// FP32 accumulation in tensor memory - the precision form of the decoder
// MLPs (Eq. 3).  Covariance, projection and blending stay float32.
//
// One CTA (8 warps) takes tiles of 128 visible anchors:
//   TMA      features of the 128 anchors (a compact BF16 copy made by
//            k_gather_bf16) arrive as four 8-column boxes, each exactly one
//            K-column of 8x16-byte core matrices of the no-swizzle K-major
//            operand layout; the view direction column is written by threads
//   MMA1     D1[128 x 96] = X[128 x 48] W1cat^T       (3 x K=16, TMEM cols 0-95)
//   epi 1    H = bf16(ReLU(D1 + b1)) into shared memory, same operand layout
//   MMA2     D2[128 x 160] = H[128 x 96] W2bd^T       (6 x K=16, TMEM cols 96-255)
//            W2bd is block diagonal by head and ordered Gaussian-major:
//            row 16j + u holds output u of Gaussian j (u = 0 opacity, 1-3
//            colour, 4-10 covariance), so a Gaussian's 11 outputs are 11
//            consecutive TMEM columns
//   epi 2    each thread owns one anchor row (TMEM lane) and five of its
//            Gaussians: activations, EWA projection, tile count, records.
// Every mbarrier wait is bounded; on a timeout the CTA flags ERR_TIMEOUT,
// drains its outstanding async work (bounded) and frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstring>
#include <vector>

#include "derive_common.cuh"

namespace gsc {

constexpr int TC_NT = 256;
constexpr int TC_M = 128;
// shared-memory image offsets (bytes)
constexpr uint32_t TC_A = 0;                        // X: 6 K-chunks x 128 rows x 16 B
constexpr uint32_t TC_W1 = TC_A + 6 * 2048;         // W1cat: 6 K-chunks x 96 rows x 16 B
constexpr uint32_t TC_W2 = TC_W1 + 6 * 1536;        // W2bd: 12 K-chunks x 160 rows x 16 B
constexpr uint32_t TC_H = TC_W2 + 12 * 2560;        // H: 12 K-chunks x 128 rows x 16 B
constexpr uint32_t TC_B1 = TC_H + 12 * 2048;        // b1 fp32 [96]
constexpr uint32_t TC_B2 = TC_B1 + 96 * 4;          // b2 fp32 [160] (Gaussian-major)
constexpr uint32_t TC_META = TC_B2 + 160 * 4;
constexpr uint32_t TC_BAR = TC_META + TC_M * 8 * 4;  // 2 mbarriers + TMEM address
// 84 KB (+ 9 KB static): two CTAs per SM, 2 x 256 = 512 TMEM columns, so a
// CTA's allocation never waits
constexpr uint32_t TC_SMEM = 84 * 1024;
static_assert(TC_BAR + 32 <= TC_SMEM, "shared-memory image exceeds the allocation");
constexpr uint32_t TC_TMEM_COLS = 256;
constexpr uint32_t TC_SPIN = 1u << 22;

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t i = 0; i < TC_SPIN; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, no swizzle, K-major: lbo = byte stride
// between core matrices along K, sbo = along M/N; version 1 (Blackwell).
__device__ __forceinline__ uint64_t make_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// Instruction descriptor, kind::f16: D f32, A/B bf16, both K-major.
__host__ __device__ constexpr uint32_t make_idesc_bf16(uint32_t M, uint32_t N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&p);
}

// ------------------------------------------------------------------ gather
// Compact BF16 features of this model's visible anchors, in the model-local
// item order of the derivation kernel (rows of 64 bytes, the TMA source).
__global__ void k_gather_bf16(const ModelDev* __restrict__ models, int model, const FrameDev* __restrict__ fd,
                              uint32_t* const* __restrict__ vis, uint4* __restrict__ out,
                              const CacheDev* __restrict__ caches) {
  __shared__ DViewSet S;
  if (threadIdx.x == 0) build_dview_set(S, fd, model, caches);
  __syncthreads();
  const uint4* src = reinterpret_cast<const uint4*>(models[model].feat_bf16);
  const uint32_t total = S.base[S.nd];
  for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < total * 4u; u += gridDim.x * blockDim.x) {
    const uint32_t item = u >> 2, part = u & 3u;
    int ld = 0;
    while (item >= S.base[ld + 1]) ++ld;
    const uint32_t w = item - S.base[ld];
    const uint32_t vi = S.miss[ld] ? S.miss[ld][w] : w;
    const uint32_t a = vis[S.d[ld]][vi];
    out[u] = src[(size_t)a * 4 + part];
  }
}

// ------------------------------------------------------------------ derivation
__global__ void __launch_bounds__(TC_NT, 1) k_derive_tc(const ModelDev* __restrict__ models, int model,
                                                        FrameDev* __restrict__ fd, uint32_t* const* __restrict__ vis,
                                                        float4* __restrict__ attrs, float* const* __restrict__ dbg_attrs,
                                                        const CacheDev* __restrict__ caches,
                                                        const __grid_constant__ CUtensorMap tmap_feat) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ DViewSet S;
  uint32_t* m_anchor = reinterpret_cast<uint32_t*>(smem + TC_META);
  uint32_t* m_vi = m_anchor + TC_M;
  int* m_ld = reinterpret_cast<int*>(m_vi + TC_M);
  float* m_pos = reinterpret_cast<float*>(m_ld + TC_M);  // [3][128]
  float* m_sa = m_pos + 3 * TC_M;
  const float* s_b1 = reinterpret_cast<const float*>(smem + TC_B1);
  const float* s_b2 = reinterpret_cast<const float*>(smem + TC_B2);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + TC_BAR);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + TC_BAR + 16);
  const uint32_t tma_bar = smem_u32(bars), mma_bar = smem_u32(bars + 1);
  const uint32_t sbase = smem_u32(smem);

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const ModelDev md = models[model];
  {  // weights image (bf16 operands, zeroed H staging area, fp32 biases), 65,536 bytes
    const uint4* src = reinterpret_cast<const uint4*>(md.w_tc);
    uint4* dst = reinterpret_cast<uint4*>(smem + TC_W1);
    for (int i = t; i < (int)((TC_META - TC_W1) / 16); i += TC_NT) dst[i] = src[i];
    // K-chunk 5 of X (K 40..47) is always zero; chunk 4 holds the direction
    uint4* z5 = reinterpret_cast<uint4*>(smem + TC_A + 5 * 2048);
    if (t < TC_M) z5[t] = make_uint4(0, 0, 0, 0);
  }
  if (t == 0) {
    build_dview_set(S, fd, model, caches);
    mbar_init(tma_bar, 1);
    mbar_init(mma_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int nd = S.nd;
  const uint32_t total = S.base[nd];
  const uint32_t ntiles = (total + TC_M - 1) / TC_M;
  const uint32_t rec_cap = fd->n_records;
  constexpr uint32_t IDESC1 = make_idesc_bf16(128, 96);
  constexpr uint32_t IDESC2 = make_idesc_bf16(128, 160);
  uint32_t tma_phase = 0, mma_phase = 0;
  bool failed = false;
  bool tma_pending = false, mma_pending = false;

  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // ---- metadata, view direction (K-chunk 4), TMA of the features (K-chunks 0-3)
    if (t < TC_M) {
      const uint32_t item = tile * TC_M + t;
      int ld = -1;
      float dx = 0.f, dy = 0.f, dz = 0.f;
      if (item < total) {
        ld = 0;
        while (item >= S.base[ld + 1]) ++ld;
        const uint32_t w = item - S.base[ld];
        const uint32_t vi = S.miss[ld] ? S.miss[ld][w] : w;
        const uint32_t a = vis[S.d[ld]][vi];
        m_anchor[t] = a;
        m_vi[t] = vi;
        const float xa = __ldg(md.px + a), ya = __ldg(md.py + a), za = __ldg(md.pz + a);
        m_pos[t] = xa; m_pos[TC_M + t] = ya; m_pos[2 * TC_M + t] = za;
        m_sa[t] = __ldg(md.scale + a);
        dx = (xa - S.pc[ld][0]) - S.pc[ld][3];
        dy = (ya - S.pc[ld][1]) - S.pc[ld][4];
        dz = (za - S.pc[ld][2]) - S.pc[ld][5];
        const float vn = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
        dx *= vn; dy *= vn; dz *= vn;
      }
      m_ld[t] = ld;
      reinterpret_cast<uint4*>(smem + TC_A + 4 * 2048)[t] = make_uint4(pack_bf16x2(dx, dy), pack_bf16x2(dz, 0.f), 0u, 0u);
      fence_proxy_async();
    }
    if (t == 0) {
      mbar_expect_tx(tma_bar, 4 * 2048);
#pragma unroll
      for (int c = 0; c < 4; ++c) tma_load_2d(sbase + TC_A + c * 2048, &tmap_feat, 8 * c, (int)(tile * TC_M), tma_bar);
    }
    tma_pending = true;
    __syncthreads();
    bool ok = mbar_wait(tma_bar, tma_phase);
    tma_phase ^= 1;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tma_pending = false;
    tc_fence_after();
    // ---- MMA1
    if (t == 0) {
#pragma unroll
      for (int ks = 0; ks < 3; ++ks)
        mma_bf16(tmem, make_sdesc(sbase + TC_A + ks * 4096, 2048, 128), make_sdesc(sbase + TC_W1 + ks * 3072, 1536, 128),
                 IDESC1, ks > 0 ? 1u : 0u);
      mma_commit(mma_bar);
    }
    mma_pending = true;
    ok = mbar_wait(mma_bar, mma_phase);
    mma_phase ^= 1;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    mma_pending = false;
    tc_fence_after();
    // ---- epilogue 1: H = bf16(ReLU(D1 + b1)); warps w and w+4 share lanes 32(w%4).., 48 columns each
    {
      const int q = warp & 3, half = warp >> 2, row = 32 * q + lane;
      const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(48 * half);
      float v[16];
#pragma unroll
      for (int g = 0; g < 3; ++g) {
        tmem_ld16(taddr + 16 * g, v);
        const int c0 = 48 * half + 16 * g;
        uint32_t pk[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          pk[u] = pack_bf16x2(fmaxf(v[2 * u] + s_b1[c0 + 2 * u], 0.f), fmaxf(v[2 * u + 1] + s_b1[c0 + 2 * u + 1], 0.f));
        uint4* h0 = reinterpret_cast<uint4*>(smem + TC_H + (c0 / 8) * 2048 + row * 16);
        uint4* h1 = reinterpret_cast<uint4*>(smem + TC_H + (c0 / 8 + 1) * 2048 + row * 16);
        *h0 = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        *h1 = make_uint4(pk[4], pk[5], pk[6], pk[7]);
      }
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // ---- MMA2
    if (t == 0) {
#pragma unroll
      for (int ks = 0; ks < 6; ++ks)
        mma_bf16(tmem + 96, make_sdesc(sbase + TC_H + ks * 4096, 2048, 128),
                 make_sdesc(sbase + TC_W2 + ks * 5120, 2560, 128), IDESC2, ks > 0 ? 1u : 0u);
      mma_commit(mma_bar);
    }
    mma_pending = true;
    ok = mbar_wait(mma_bar, mma_phase);
    mma_phase ^= 1;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    mma_pending = false;
    tc_fence_after();
    // ---- epilogue 2: one anchor row per thread, five Gaussians per thread
    {
      const int q = warp & 3, half = warp >> 2, row = 32 * q + lane;
      const int ld = m_ld[row];
      const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16) + 96u;
#pragma unroll 1
      for (int jj = 0; jj < 5; ++jj) {
        const int j = 5 * half + jj;
        float v[16];
        tmem_ld16(trow + 16 * j, v);  // all lanes: .sync.aligned
        if (ld < 0) continue;
        float z[11];
#pragma unroll
        for (int u = 0; u < 11; ++u) z[u] = v[u] + s_b2[16 * j + u];
        float* dbg = dbg_attrs ? dbg_attrs[S.d[ld]] : nullptr;
        const size_t idx = (size_t)(S.gbase[ld] + m_vi[row]) * K + j;
        uint2* line = nullptr;
        if (S.vstat[ld]) {
          const uint32_t st = S.vstat[ld][m_vi[row]];
          if (st != LINE_NONE && !(st & LINE_HIT)) line = S.lattr[ld] + ((size_t)st * K + j) * 3;
        }
        if (idx < rec_cap) gaussian_activate_store(z, j, m_vi[row], m_sa[row], attrs, idx, dbg, line);
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  if (failed) {
    if (t == 0) atomicOr(&fd->err, ERR_TIMEOUT);
    // drain what may still be in flight (bounded) before the memory goes away
    if (tma_pending) (void)mbar_wait(tma_bar, tma_phase ^ 1);
    if (mma_pending) (void)mbar_wait(mma_bar, mma_phase ^ 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
}

cudaError_t prepare_derive_tc() {
  return cudaFuncSetAttribute(k_derive_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
}

__global__ void k_to_bf16(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

void launch_to_bf16(const float* src, void* dst, size_t n, cudaStream_t s) {
  if (n) k_to_bf16<<<1024, 256, 0, s>>>(src, static_cast<__nv_bfloat16*>(dst), n);
}

// Tensor map of the compact feature buffer: rows of 32 bf16, boxes of 8
// columns x 128 rows (one K-chunk of core matrices per box).
int encode_feat_tmap(CUtensorMap* map, void* base, uint64_t rows) {
  using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
      return -1;
    fn = reinterpret_cast<EncodeFn>(p);
  }
  const cuuint64_t dims[2] = {32, rows};
  const cuuint64_t strides[1] = {64};
  const cuuint32_t box[2] = {8, 128};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -1;
}

// bf16 round-to-nearest-even of a float (host side, for the weight image).
static uint16_t host_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

// The 65,536-byte shared-memory image of the tensor-core MLP weights:
// W1cat as the B operand [96 rows (hidden) x 48 K] and the Gaussian-major
// block-diagonal W2 as the B operand [160 rows x 96 K], both in K-chunks of
// 8 bf16 x all rows (16 bytes per row), the hidden-activation staging area
// (zeros here), then b1 [96] and b2 [160] in fp32.
void pack_tc_weights(const float* const W1[3], const float* const b1[3], const float* const W2[3],
                     const float* const b2[3], std::vector<uint8_t>& img) {
  img.assign(TC_META - TC_W1, 0);
  uint16_t* w1 = reinterpret_cast<uint16_t*>(img.data());
  uint16_t* w2 = reinterpret_cast<uint16_t*>(img.data() + (TC_W2 - TC_W1));
  float* fb1 = reinterpret_cast<float*>(img.data() + (TC_B1 - TC_W1));
  float* fb2 = reinterpret_cast<float*>(img.data() + (TC_B2 - TC_W1));
  for (int k = 0; k < IN; ++k)
    for (int n = 0; n < NH; ++n) w1[(k / 8) * (1536 / 2) + n * 8 + (k % 8)] = host_bf16(W1[n / HID][k * HID + n % HID]);
  for (int n = 0; n < NH; ++n) fb1[n] = b1[n / HID][n % HID];
  const int outd[3] = {K, 3 * K, 7 * K};
  for (int j = 0; j < K; ++j)
    for (int u = 0; u < 11; ++u) {
      const int head = u == 0 ? 0 : (u < 4 ? 1 : 2);
      const int out = u == 0 ? j : (u < 4 ? 3 * j + u - 1 : 7 * j + u - 4);
      const int n = 16 * j + u;
      for (int c = 0; c < HID; ++c) {
        const int k = head * HID + c;
        w2[(k / 8) * (2560 / 2) + n * 8 + (k % 8)] = host_bf16(W2[head][c * outd[head] + out]);
      }
      fb2[n] = b2[head][out];
    }
}

void launch_derive_tc(const ModelDev* models, int model, FrameDev* fd, uint32_t* const* vis, float4* attrs,
                      float* const* dbg_attrs, const CacheDev* caches, const CUtensorMap* tmap, uint4* compact,
                      int n_sm, cudaStream_t s) {
  k_gather_bf16<<<n_sm * 4, 256, 0, s>>>(models, model, fd, vis, compact, caches);
  k_derive_tc<<<n_sm * 2, TC_NT, TC_SMEM, s>>>(models, model, fd, vis, attrs, dbg_attrs, caches, *tmap);
}

}  // namespace gsc
