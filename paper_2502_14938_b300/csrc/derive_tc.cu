// Derivation on the 5th-generation tensor cores (tcgen05), BF16 or FP8-E4M3
// inputs with FP32 accumulation in tensor memory - the precision forms of
// the decoder MLPs (Eq. 3).  Covariance, projection and blending stay float32.
// FP8 uses per-tensor power-of-two scales (inputs, each head's W1 / W2 and
// hidden layer): the accumulators are multiplied back by s_x s_w1 (layer 1)
// and s_h s_w2 (layer 2), the hidden layer is divided by s_h before it is
// rounded to E4M3.  The weights and the hidden activations are two-term E4M3
// expansions at their scale (hi, and lo = e4m3(value - hi)): layer 1 adds the
// MMAs with W1_lo, layer 2 those of H_lo x W2 and H x W2_lo, into the same
// FP32 accumulators; the inputs stay one E4M3 term.  Operand tiles are the
// same 16-byte core matrices either way: 8 bf16 or 16 e4m3 per K-chunk, K =
// 16 or 32 per MMA.
//
// One CTA (8 warps) takes tiles of 128 visible anchors:
//   load     thread t < 128 fetches row t: the anchor's id, position, scale
//            and line status and, in the same round trip, its feature row
//            straight from the model's BF16 (E4M3) feature table (16-byte
//            vector loads), stored as K-columns of 8x16-byte core matrices of
//            the no-swizzle K-major operand layout; the view direction
//            column likewise
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
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "derive_common.cuh"

namespace gsc {

constexpr int TC_NT = 256;
constexpr int TC_M = 128;
// Shared-memory image of one CTA (bytes).  X: XCH K-chunks x 128 rows x 16 B;
// W1cat: XCH x 96 rows; W2bd: HCH x 160 rows; H: HCH x 128 rows (FP8: each
// of W1, W2 and H followed by its second term, same size); then fp32 b1 [96]
// (FP8: + s1 [96] dequant, r1 [96] 1/s_h), b2 [160] (FP8: + s2 [160]
// dequant), per-row metadata, 2 mbarriers and the TMEM address.
template <bool FP8>
struct TcL {
  static constexpr int XCH = FP8 ? 4 : 6, HCH = FP8 ? 6 : 12;
  static constexpr int K1 = FP8 ? 2 : 3, K2 = FP8 ? 3 : 6;  // MMA K-steps
  static constexpr int FEAT_CH = FP8 ? 2 : 4;                 // feature chunks (16 B of a row each)
  static constexpr int DIR_CH = FP8 ? 2 : 4;                  // direction chunk
  static constexpr int ZERO_CH = FP8 ? 3 : 5;                 // always-zero chunk
  static constexpr uint32_t A = 0;
  static constexpr uint32_t W1 = A + XCH * 2048;
  static constexpr uint32_t W1LO = W1 + XCH * 1536;
  static constexpr uint32_t W2 = W1LO + (FP8 ? XCH * 1536 : 0);
  static constexpr uint32_t W2LO = W2 + HCH * 2560;
  static constexpr uint32_t H = W2LO + (FP8 ? HCH * 2560 : 0);
  static constexpr uint32_t HLO = H + HCH * 2048;
  static constexpr uint32_t B1 = HLO + (FP8 ? HCH * 2048 : 0);
  static constexpr uint32_t S1 = B1 + 96 * 4;
  static constexpr uint32_t R1 = S1 + 96 * 4;
  static constexpr uint32_t B2 = FP8 ? R1 + 96 * 4 : S1;
  static constexpr uint32_t S2 = B2 + 160 * 4;
  static constexpr uint32_t META = FP8 ? S2 + 160 * 4 : S2;
  static constexpr uint32_t BAR = META + TC_M * 8 * 4;
  static constexpr uint32_t IMG = META - W1;  // bytes of the weight image
};
// 84 KB (+ 9 KB static): two CTAs per SM, 2 x 256 = 512 TMEM columns, so a
// CTA's allocation never waits
constexpr uint32_t TC_SMEM = 84 * 1024;
// BAR: mbarriers for the features (+0) and the MMAs (+8), TMEM address (+16),
// mbarrier for the weight image (+24)
static_assert(TcL<false>::BAR + 32 <= TC_SMEM && TcL<true>::BAR + 32 <= TC_SMEM,
              "shared-memory image exceeds the allocation");
static_assert(TcL<false>::IMG == 65536 && TcL<true>::IMG == 70016, "weight image sizes");
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
// Untiled bulk copy global -> shared (both 16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
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
// Instruction descriptors, D f32, A and B K-major: kind::f16 with A/B bf16
// (format 1 at bits 7 and 10); kind::f8f6f4 with A/B e4m3 (format 0).
__host__ __device__ constexpr uint32_t make_idesc_bf16(uint32_t M, uint32_t N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}
__host__ __device__ constexpr uint32_t make_idesc_e4m3(uint32_t M, uint32_t N) {
  return (1u << 4) | ((N >> 3) << 17) | ((M >> 4) << 24);
}
template <bool FP8>
__device__ __forceinline__ void mma_tc(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  if constexpr (FP8)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::
            "r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::
            "r"(tmem_d),
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
// Four e4m3 bytes (element 0 lowest) -> four floats.
__device__ __forceinline__ void unpack_e4m3x4(uint32_t v, float out[4]) {
  const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(v & 0xFFFFu), __NV_E4M3);
  const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(v >> 16), __NV_E4M3);
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&lo));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&hi));
  out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
}

// Four floats -> four e4m3 bytes (round to nearest even, saturating), element 0 lowest.
__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d) {
  const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
  const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
  return (lo & 0xFFFFu) | (hi << 16);
}

// ------------------------------------------------------------------ derivation
template <bool FP8>
__global__ void __launch_bounds__(TC_NT, 1) k_derive_tc(const ModelDev* __restrict__ models, int model,
                                                        FrameDev* __restrict__ fd, uint32_t* const* __restrict__ vis,
                                                        float4* __restrict__ attrs, float* const* __restrict__ dbg_attrs,
                                                        const CacheDev* __restrict__ caches,
                                                        const DViewSet* __restrict__ tabs) {
  using L = TcL<FP8>;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ DViewSet S;
  uint32_t* m_anchor = reinterpret_cast<uint32_t*>(smem + L::META);
  uint32_t* m_vi = m_anchor + TC_M;
  int* m_ld = reinterpret_cast<int*>(m_vi + TC_M);
  float* m_pos = reinterpret_cast<float*>(m_ld + TC_M);  // [3][128]
  float* m_sa = m_pos + 3 * TC_M;
  uint32_t* m_line = reinterpret_cast<uint32_t*>(m_sa + TC_M);  // line to write, or LINE_NONE
  const float* s_b1 = reinterpret_cast<const float*>(smem + L::B1);
  const float* s_s1 = reinterpret_cast<const float*>(smem + L::S1);
  const float* s_r1 = reinterpret_cast<const float*>(smem + L::R1);
  const float* s_b2 = reinterpret_cast<const float*>(smem + L::B2);
  const float* s_s2 = reinterpret_cast<const float*>(smem + L::S2);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::BAR);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::BAR + 16);
  const uint32_t mma_bar = smem_u32(bars + 1);
  const uint32_t sbase = smem_u32(smem);

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const ModelDev md = models[model];
  load_dview_set(S, tabs, fd, model, caches);
  if (blockIdx.x >= (S.base[S.nd] + TC_M - 1) / TC_M) return;  // no tile: skip weights, barriers and TMEM
  const uint32_t w_bar = smem_u32(bars + 3);  // weight image barrier (after the TMEM address slot)
  {  // the last K-chunk of X is always zero; the one before holds the direction
    uint4* zc = reinterpret_cast<uint4*>(smem + L::A + L::ZERO_CH * 2048);
    if (t < TC_M) zc[t] = make_uint4(0, 0, 0, 0);
  }
  if (t == 0) {
    mbar_init(mma_bar, 1);
    mbar_init(w_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // weights image (operands, zeroed H staging area, fp32 biases and scales): one bulk copy
    mbar_expect_tx(w_bar, L::IMG);
    bulk_load(sbase + L::W1, FP8 ? md.w_tc8 : md.w_tc, L::IMG, w_bar);
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
  constexpr uint32_t IDESC1 = FP8 ? make_idesc_e4m3(128, 96) : make_idesc_bf16(128, 96);
  constexpr uint32_t IDESC2 = FP8 ? make_idesc_e4m3(128, 160) : make_idesc_bf16(128, 160);
  uint32_t mma_phase = 0;
  bool failed = false;
  bool mma_pending = false;
  bool w_pending = true;  // the weight image is waited for just before the first MMA, so that its
                          // copy overlaps the first tile's metadata and feature loads

  for (uint32_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    // ---- metadata, view direction chunk, feature chunks
    if (t < TC_M) {  // thread t: row t's metadata, view direction and feature chunks
      const uint32_t item = tile * TC_M + t;
      int ld = -1;
      uint32_t a = 0, vi = 0, line = LINE_NONE;  // rows past the end load anchor 0; nothing is stored
      if (item < total) {
        ld = 0;
        while (item >= S.base[ld + 1]) ++ld;
        const uint32_t w = item - S.base[ld];
        vi = S.miss[ld] ? S.miss[ld][w] : w;
        a = vis[S.d[ld]][vi];
        if (S.vstat[ld]) {  // a miss with a line (refresh or new) rewrites it
          const uint32_t st = S.vstat[ld][vi];
          if (st != LINE_NONE && !(st & LINE_HIT)) line = st;
        }
      }
      // the feature row (16-byte K-chunks into the operand layout) is
      // fetched beside the position and scale: one round trip for both
      const uint4* ft = reinterpret_cast<const uint4*>(FP8 ? md.feat_fp8 : md.feat_bf16) + (size_t)a * L::FEAT_CH;
      uint4 fc[L::FEAT_CH];
#pragma unroll
      for (int c = 0; c < L::FEAT_CH; ++c) fc[c] = __ldg(ft + c);
      float dx = 0.f, dy = 0.f, dz = 0.f;
      if (ld >= 0) {
        const float xa = __ldg(md.px + a), ya = __ldg(md.py + a), za = __ldg(md.pz + a);
        m_pos[t] = xa; m_pos[TC_M + t] = ya; m_pos[2 * TC_M + t] = za;
        m_sa[t] = __ldg(md.scale + a);
        dx = (xa - S.pc[ld][0]) - S.pc[ld][3];
        dy = (ya - S.pc[ld][1]) - S.pc[ld][4];
        dz = (za - S.pc[ld][2]) - S.pc[ld][5];
        const float vn = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
        dx *= vn; dy *= vn; dz *= vn;
      }
      m_anchor[t] = a;
      m_vi[t] = vi;
      m_line[t] = line;
      m_ld[t] = ld;
#pragma unroll
      for (int c = 0; c < L::FEAT_CH; ++c) reinterpret_cast<uint4*>(smem + L::A + c * 2048)[t] = fc[c];
      uint4 dirc;
      if constexpr (FP8) {
        const float ix = md.fp8_inv_sx;  // 1 / s_x, a power of two
        dirc = make_uint4(pack_e4m3x4(dx * ix, dy * ix, dz * ix, 0.f), 0u, 0u, 0u);
      } else {
        dirc = make_uint4(pack_bf16x2(dx, dy), pack_bf16x2(dz, 0.f), 0u, 0u);
      }
      reinterpret_cast<uint4*>(smem + L::A + L::DIR_CH * 2048)[t] = dirc;
      fence_proxy_async();  // generic-proxy writes, read by the MMA's async proxy
    }
    __syncthreads();  // the tile's rows
    if (w_pending) {
      if (__syncthreads_or(!mbar_wait(w_bar, 0))) {
        failed = true;
        break;
      }
      w_pending = false;
    }
    tc_fence_after();
    // ---- MMA1
    if (t == 0) {
#pragma unroll
      for (int ks = 0; ks < L::K1; ++ks)
        mma_tc<FP8>(tmem, make_sdesc(sbase + L::A + ks * 4096, 2048, 128),
                    make_sdesc(sbase + L::W1 + ks * 3072, 1536, 128), IDESC1, ks > 0 ? 1u : 0u);
      if constexpr (FP8) {  // + X W1_lo
#pragma unroll
        for (int ks = 0; ks < L::K1; ++ks)
          mma_tc<FP8>(tmem, make_sdesc(sbase + L::A + ks * 4096, 2048, 128),
                      make_sdesc(sbase + L::W1LO + ks * 3072, 1536, 128), IDESC1, 1u);
      }
      mma_commit(mma_bar);
    }
    mma_pending = true;
    bool ok = mbar_wait(mma_bar, mma_phase);
    mma_phase ^= 1;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    mma_pending = false;
    tc_fence_after();
    // ---- epilogue 1: H = ReLU(D1 + b1) (FP8: D1 s_x s_w1 + b1, then / s_h)
    // rounded to the operand type; warps w and w+4 share lanes 32(w%4).., 48 columns each
    {
      const int q = warp & 3, half = warp >> 2, row = 32 * q + lane;
      const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(48 * half);
      float v[16];
#pragma unroll
      for (int g = 0; g < 3; ++g) {
        tmem_ld16(taddr + 16 * g, v);
        const int c0 = 48 * half + 16 * g;
        if constexpr (FP8) {
          float h[16];
#pragma unroll
          for (int u = 0; u < 16; ++u) h[u] = fmaxf(fmaf(v[u], s_s1[c0 + u], s_b1[c0 + u]), 0.f) * s_r1[c0 + u];
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {  // h = hi + lo: lo rounds the (exact) residual h - hi
            hi[u] = pack_e4m3x4(h[4 * u], h[4 * u + 1], h[4 * u + 2], h[4 * u + 3]);
            float r[4];
            unpack_e4m3x4(hi[u], r);
            lo[u] = pack_e4m3x4(h[4 * u] - r[0], h[4 * u + 1] - r[1], h[4 * u + 2] - r[2], h[4 * u + 3] - r[3]);
          }
          *reinterpret_cast<uint4*>(smem + L::H + (c0 / 16) * 2048 + row * 16) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<uint4*>(smem + L::HLO + (c0 / 16) * 2048 + row * 16) =
              make_uint4(lo[0], lo[1], lo[2], lo[3]);
        } else {
          uint32_t pk[8];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            pk[u] = pack_bf16x2(fmaxf(v[2 * u] + s_b1[c0 + 2 * u], 0.f), fmaxf(v[2 * u + 1] + s_b1[c0 + 2 * u + 1], 0.f));
          uint4* h0 = reinterpret_cast<uint4*>(smem + L::H + (c0 / 8) * 2048 + row * 16);
          uint4* h1 = reinterpret_cast<uint4*>(smem + L::H + (c0 / 8 + 1) * 2048 + row * 16);
          *h0 = make_uint4(pk[0], pk[1], pk[2], pk[3]);
          *h1 = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
      }
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // ---- MMA2
    if (t == 0) {
#pragma unroll
      for (int ks = 0; ks < L::K2; ++ks)
        mma_tc<FP8>(tmem + 96, make_sdesc(sbase + L::H + ks * 4096, 2048, 128),
                    make_sdesc(sbase + L::W2 + ks * 5120, 2560, 128), IDESC2, ks > 0 ? 1u : 0u);
      if constexpr (FP8) {  // + H_lo W2 + H W2_lo
#pragma unroll
        for (int ks = 0; ks < L::K2; ++ks) {
          mma_tc<FP8>(tmem + 96, make_sdesc(sbase + L::HLO + ks * 4096, 2048, 128),
                      make_sdesc(sbase + L::W2 + ks * 5120, 2560, 128), IDESC2, 1u);
          mma_tc<FP8>(tmem + 96, make_sdesc(sbase + L::H + ks * 4096, 2048, 128),
                      make_sdesc(sbase + L::W2LO + ks * 5120, 2560, 128), IDESC2, 1u);
        }
      }
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
      const uint32_t vi = m_vi[row], mline = m_line[row];
      const float sa = m_sa[row];
      float* dbg = ld >= 0 && dbg_attrs ? dbg_attrs[S.d[ld]] : nullptr;
      const size_t idx0 = ld >= 0 ? (size_t)(S.gbase[ld] + vi) * K : 0;
      uint2* lbase = ld >= 0 && mline != LINE_NONE ? S.lattr[ld] + (size_t)mline * K * 3 : nullptr;
      const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16) + 96u;
#pragma unroll 1
      for (int jj = 0; jj < 5; ++jj) {
        const int j = 5 * half + jj;
        float v[16];
        tmem_ld16(trow + 16 * j, v);  // all lanes: .sync.aligned
        if (ld < 0) continue;
        float z[11];
#pragma unroll
        for (int u = 0; u < 11; ++u) z[u] = FP8 ? fmaf(v[u], s_s2[16 * j + u], s_b2[16 * j + u]) : v[u] + s_b2[16 * j + u];
        const size_t idx = idx0 + j;
        uint2* line = lbase ? lbase + (size_t)j * 3 : nullptr;
        if (idx < rec_cap) gaussian_activate_store<true>(z, j, vi, sa, attrs, idx, dbg, line);
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  if (failed) {
    if (t == 0) atomicOr(&fd->err, ERR_TIMEOUT);
    // drain what may still be in flight (bounded) before the memory goes away
    if (w_pending) (void)mbar_wait(w_bar, 0);
    if (mma_pending) (void)mbar_wait(mma_bar, mma_phase ^ 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
}

cudaError_t prepare_derive_tc() {
  cudaError_t e = cudaFuncSetAttribute(k_derive_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_derive_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
}

__global__ void k_to_bf16(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

void launch_to_bf16(const float* src, void* dst, size_t n, cudaStream_t s) {
  if (n) k_to_bf16<<<1024, 256, 0, s>>>(src, static_cast<__nv_bfloat16*>(dst), n);
}

// e4m3(x * inv_scale), round to nearest even, saturating.
__global__ void k_to_e4m3(const float* __restrict__ src, float inv_scale, uint8_t* __restrict__ dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (uint8_t)__nv_cvt_float_to_fp8(src[i] * inv_scale, __NV_SATFINITE, __NV_E4M3);
}

void launch_to_e4m3(const float* src, float inv_scale, void* dst, size_t n, cudaStream_t s) {
  if (n) k_to_e4m3<<<1024, 256, 0, s>>>(src, inv_scale, static_cast<uint8_t*>(dst), n);
}

// Two-term e4m3 expansion: hi = e4m3(x), lo = e4m3(x - hi) (the residual is
// exact in float32), round to nearest even, saturating.
__global__ void k_to_e4m3_two_term(const float* __restrict__ src, uint8_t* __restrict__ hi, uint8_t* __restrict__ lo,
                                   size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float x = src[i];
    const __nv_fp8_storage_t h = __nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
    const __half_raw hr = __nv_cvt_fp8_to_halfraw(h, __NV_E4M3);
    const float hf = __half2float(*reinterpret_cast<const __half*>(&hr));
    hi[i] = (uint8_t)h;
    lo[i] = (uint8_t)__nv_cvt_float_to_fp8(x - hf, __NV_SATFINITE, __NV_E4M3);
  }
}

void launch_to_e4m3_two_term(const float* src, void* hi, void* lo, size_t n, cudaStream_t s) {
  if (n)
    k_to_e4m3_two_term<<<256, 256, 0, s>>>(src, static_cast<uint8_t*>(hi), static_cast<uint8_t*>(lo), n);
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
  using L = TcL<false>;
  img.assign(L::IMG, 0);
  uint16_t* w1 = reinterpret_cast<uint16_t*>(img.data());
  uint16_t* w2 = reinterpret_cast<uint16_t*>(img.data() + (L::W2 - L::W1));
  float* fb1 = reinterpret_cast<float*>(img.data() + (L::B1 - L::W1));
  float* fb2 = reinterpret_cast<float*>(img.data() + (L::B2 - L::W1));
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

// ------------------------------------------------------------------ FP8 form
namespace {
float pow2_at_least(double v) {  // smallest power of two >= v; 1 for v <= 0
  if (!(v > 0.0)) return 1.f;
  int e;
  const double m = std::frexp(v, &e);  // v = m 2^e, m in [0.5, 1)
  return (float)std::ldexp(1.0, m == 0.5 ? e - 1 : e);
}
}  // namespace

// Per-tensor scales: amax / 448 rounded up to a power of two (exact scaling).
// Inputs: max(amax of the features, 1) (the unit direction shares the input
// tensor); hidden layer: max over units o of sum_c |W1[c][o]| amax_c + |b1[o]|,
// a bound over every anchor and view direction (amax_c: largest |feature c|,
// 1 for a direction component).
Fp8Scales fp8_scales(const float* feat, size_t n, const float* const W1[3], const float* const b1[3],
                     const float* const W2[3]) {
  Fp8Scales S{};
  double amax_c[IN];
  for (int c = 0; c < IN; ++c) amax_c[c] = c < FDIM ? 0.0 : 1.0;
  for (size_t a = 0; a < n; ++a)
    for (int c = 0; c < FDIM; ++c) amax_c[c] = std::max(amax_c[c], (double)std::fabs(feat[a * FDIM + c]));
  double ax = 1.0;
  for (int c = 0; c < FDIM; ++c) ax = std::max(ax, amax_c[c]);
  S.sx = pow2_at_least(ax / 448.0);
  const int outd[3] = {K, 3 * K, 7 * K};
  for (int h = 0; h < 3; ++h) {
    double a1 = 0.0, a2 = 0.0, hb = 0.0;
    for (int i = 0; i < IN * HID; ++i) a1 = std::max(a1, (double)std::fabs(W1[h][i]));
    for (int i = 0; i < HID * outd[h]; ++i) a2 = std::max(a2, (double)std::fabs(W2[h][i]));
    for (int o = 0; o < HID; ++o) {
      double b = std::fabs((double)b1[h][o]);
      for (int c = 0; c < IN; ++c) b += std::fabs((double)W1[h][c * HID + o]) * amax_c[c];
      hb = std::max(hb, b);
    }
    S.sw1[h] = pow2_at_least(a1 / 448.0);
    S.sw2[h] = pow2_at_least(a2 / 448.0);
    S.sh[h] = pow2_at_least(hb / 448.0);
  }
  return S;
}

// The 70,016-byte FP8 image (layout TcL<true>): e4m3 W1cat [96 x 64 K] and
// its second term, block-diagonal W2bd [160 x 96 K] and its second term
// (each weight divided by its head's scale, split on the device), the
// zeroed H and H_lo areas, then fp32 b1, s1 = s_x s_w1, r1 = 1 / s_h per
// hidden unit and b2, s2 = s_h s_w2 per output row.
cudaError_t make_tc8_image(const float* const W1[3], const float* const b1[3], const float* const W2[3],
                           const float* const b2[3], const Fp8Scales& S, void* d_img, cudaStream_t s) {
  using L = TcL<true>;
  const size_t n_w1 = L::XCH * 1536, n_w2 = L::HCH * 2560;
  std::vector<float> pre(n_w1 + n_w2, 0.f);
  for (int k = 0; k < IN; ++k)
    for (int n = 0; n < NH; ++n)
      pre[(k / 16) * 1536 + n * 16 + (k % 16)] = W1[n / HID][k * HID + n % HID] / S.sw1[n / HID];
  const int outd[3] = {K, 3 * K, 7 * K};
  std::vector<float> tail((L::META - L::B1) / 4, 0.f);
  float* fb1 = tail.data();
  float* fs1 = tail.data() + (L::S1 - L::B1) / 4;
  float* fr1 = tail.data() + (L::R1 - L::B1) / 4;
  float* fb2 = tail.data() + (L::B2 - L::B1) / 4;
  float* fs2 = tail.data() + (L::S2 - L::B1) / 4;
  for (int n = 0; n < NH; ++n) {
    fb1[n] = b1[n / HID][n % HID];
    fs1[n] = S.sx * S.sw1[n / HID];
    fr1[n] = 1.0f / S.sh[n / HID];
  }
  for (int j = 0; j < K; ++j)
    for (int u = 0; u < 11; ++u) {
      const int head = u == 0 ? 0 : (u < 4 ? 1 : 2);
      const int out = u == 0 ? j : (u < 4 ? 3 * j + u - 1 : 7 * j + u - 4);
      const int n = 16 * j + u;
      for (int c = 0; c < HID; ++c) {
        const int k = head * HID + c;
        pre[n_w1 + (k / 16) * 2560 + n * 16 + (k % 16)] = W2[head][c * outd[head] + out] / S.sw2[head];
      }
      fb2[n] = b2[head][out];
      fs2[n] = S.sh[head] * S.sw2[head];
    }
  float* d_pre = nullptr;
  cudaError_t e = cudaMalloc((void**)&d_pre, pre.size() * 4);
  if (e != cudaSuccess) return e;
  uint8_t* img = static_cast<uint8_t*>(d_img);
  if ((e = cudaMemcpy(d_pre, pre.data(), pre.size() * 4, cudaMemcpyHostToDevice)) == cudaSuccess) {
    launch_to_e4m3_two_term(d_pre, img + (L::W1 - L::W1), img + (L::W1LO - L::W1), n_w1, s);
    launch_to_e4m3_two_term(d_pre + n_w1, img + (L::W2 - L::W1), img + (L::W2LO - L::W1), n_w2, s);
    e = cudaStreamSynchronize(s);
  }
  cudaFree(d_pre);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemset(img + (L::H - L::W1), 0, 2 * L::HCH * 2048)) != cudaSuccess) return e;
  return cudaMemcpy(img + (L::B1 - L::W1), tail.data(), tail.size() * 4, cudaMemcpyHostToDevice);
}

void launch_derive_tc(const ModelDev* models, int model, FrameDev* fd, uint32_t* const* vis, float4* attrs,
                      float* const* dbg_attrs, const CacheDev* caches, const DViewSet* tabs, bool fp8, int n_sm,
                      cudaStream_t s) {
  if (fp8)
    k_derive_tc<true><<<n_sm * 2, TC_NT, TC_SMEM, s>>>(models, model, fd, vis, attrs, dbg_attrs, caches, tabs);
  else
    k_derive_tc<false><<<n_sm * 2, TC_NT, TC_SMEM, s>>>(models, model, fd, vis, attrs, dbg_attrs, caches, tabs);
}

}  // namespace gsc
