// Learned reuse predictor (K12): inputs and the reuse decision.
//
// The cache of Sec. 4 reuses a line by the depth rule of Alg. 1 / Eq. 4; the
// learned form replaces "age <= depth" by a small network's decision,
//   p = sigmoid(w2 . relu(W1^T z + b1) + b2),  reuse iff p >= 0.5 (logit >= 0),
// with re-derivation as the fallback.  z (36 values) of a visible anchor with
// a valid line:
//   z[0:32]  the anchor feature,
//   z[32:35] 1024 (dir_now - dir_line): change of the unit direction from the
//            derivation camera's centre to the anchor since the line was
//            decoded,
//   z[35]    plog2(|x_a - p|) - 8, plog2(m 2^e) = e + (m - 1) for m in [1, 2).
// The decision is an integer, so everything feeding it is float32 with one
// fixed operation order and no contraction (round-to-nearest intrinsics),
// weights rounded to bfloat16:
//   dx = (x_a - p_hi) - p_lo,  |dx| = sqrt((dx0 dx0 + dx1 dx1) + dx2 dx2),
//   dir = dx / |dx|,
//   h_j = max(0, (sum_k w[k][j] z_k, left to right) + b1_j),
//   logit = (sum_j w2_j h_j, left to right) + b2.
// Parameter layout (flat, float): W1 [36][64] input-major, b1 [64], w2 [64], b2.
#pragma once
#include <cuda_fp16.h>

#include "gsc_internal.cuh"

namespace gsc {

constexpr int RZ = 36;
constexpr int RH = 64;
constexpr int RPARAM = RZ * RH + RH + RH + 1;  // 2433
constexpr int R_B1 = RZ * RH, R_W2 = RZ * RH + RH, R_B2 = RZ * RH + 2 * RH;

// Unit direction and distance from the double-float centre (pc, pc_lo) to x.
__device__ __forceinline__ float pinned_dir(const float* __restrict__ x, const float pc[3], const float pc_lo[3],
                                            float d[3]) {
  float dx[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) dx[i] = __fsub_rn(__fsub_rn(x[i], pc[i]), pc_lo[i]);
  const float n2 = __fadd_rn(__fadd_rn(__fmul_rn(dx[0], dx[0]), __fmul_rn(dx[1], dx[1])), __fmul_rn(dx[2], dx[2]));
  const float n = __fsqrt_rn(n2);
#pragma unroll
  for (int i = 0; i < 3; ++i) d[i] = n > 0.f ? __fdiv_rn(dx[i], n) : 0.f;
  return n;
}

// (e - 8) + (m - 1) for n = m 2^e, m in [1, 2); n <= 0 gives -135.
__device__ __forceinline__ float plog2_m8(float n) {
  if (!(n > 0.f)) return -135.f;
  const uint32_t b = __float_as_uint(n);
  const int e = (int)((b >> 23) & 0xFFu) - 127;
  const float m = __uint_as_float((b & 0x7FFFFFu) | 0x3F800000u);
  return __fadd_rn((float)(e - 8), __fsub_rn(m, 1.0f));
}

__device__ __forceinline__ void reuse_features(const float* __restrict__ feat, const float dnow[3],
                                               const float dline[3], float dist, float z[RZ]) {
#pragma unroll
  for (int k = 0; k < FDIM; ++k) z[k] = feat[k];
#pragma unroll
  for (int i = 0; i < 3; ++i) z[FDIM + i] = __fmul_rn(__fsub_rn(dnow[i], dline[i]), 1024.0f);
  z[RZ - 1] = plog2_m8(dist);
}

// Pinned logit; w: the bfloat16-rounded parameters (as float), any address space.
__device__ __forceinline__ float reuse_logit(const float* __restrict__ w, const float z[RZ]) {
  float acc[RH];
#pragma unroll
  for (int j = 0; j < RH; ++j) acc[j] = 0.f;
#pragma unroll 4
  for (int k = 0; k < RZ; ++k) {
    const float zk = z[k];
#pragma unroll
    for (int j = 0; j < RH; ++j) acc[j] = __fadd_rn(acc[j], __fmul_rn(w[k * RH + j], zk));
  }
  float out = 0.f;
#pragma unroll
  for (int j = 0; j < RH; ++j) {
    float h = __fadd_rn(acc[j], w[R_B1 + j]);
    h = h > 0.f ? h : 0.f;
    out = __fadd_rn(out, __fmul_rn(w[R_W2 + j], h));
  }
  return __fadd_rn(out, w[R_B2]);
}

}  // namespace gsc
