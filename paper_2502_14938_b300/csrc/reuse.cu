// Training of the reuse predictor (K12) on the GPU.
//
// Mean binary cross-entropy of sigmoid(logit) against the labels, minimised
// by Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) over shuffled
// mini-batches.  Master weights are float32; the forward and backward passes
// use their bfloat16 rounding (the weights inference uses) with float32
// arithmetic.  Per mini-batch:
//   k_reuse_fwdbwd  one block of 64 threads (thread j = hidden unit j) per
//                   64 samples: hidden pre-activations, logits, d loss/d logit
//                   (p - y) / B, and the block's gradient sums, written as a
//                   partial (no atomics: the result does not depend on
//                   scheduling)
//   k_reuse_reduce  partials summed in block order -> gradient, loss
//   k_reuse_adam    moments, bias correction, update, bf16 forward copy
//   k_reuse_tick    step counter (and, once per epoch, the epoch counter)
// A whole epoch is captured as one CUDA graph and replayed; the sample order
// of epoch e is order[e * n + i], read through the device epoch counter.
#include <cuda_bf16.h>

#include "reuse_common.cuh"

namespace gsc {

constexpr int RT_CHUNK = 64;          // samples per block
constexpr int RT_NPART = RPARAM + 1;  // gradient sums + loss sum

__global__ void __launch_bounds__(RH) k_reuse_fwdbwd(const float* __restrict__ Z, const float* __restrict__ Y,
                                                     const uint32_t* __restrict__ order,
                                                     const uint32_t* __restrict__ ctl, uint32_t n_total,
                                                     uint32_t b0, uint32_t nb, float inv_nb,
                                                     const float* __restrict__ w, float* __restrict__ part) {
  __shared__ float s_z[RT_CHUNK][RZ + 1];
  __shared__ float s_h[RT_CHUNK][RH + 1];
  __shared__ float s_g[RT_CHUNK];
  __shared__ float s_l[RT_CHUNK];
  const int j = threadIdx.x;
  const uint32_t first = blockIdx.x * RT_CHUNK;
  const int ns = (int)min((uint32_t)RT_CHUNK, nb - first);
  const size_t ebase = (size_t)ctl[1] * n_total + b0 + first;
  for (int i = j; i < ns * RZ; i += RH) {
    const int s = i / RZ, k = i % RZ;
    s_z[s][k] = Z[(size_t)order[ebase + s] * RZ + k];
  }
  float wj[RZ];
#pragma unroll
  for (int k = 0; k < RZ; ++k) wj[k] = w[k * RH + j];
  const float b1j = w[R_B1 + j], w2j = w[R_W2 + j];
  __syncthreads();
  for (int s = 0; s < ns; ++s) {
    float pre = b1j;
#pragma unroll
    for (int k = 0; k < RZ; ++k) pre = fmaf(wj[k], s_z[s][k], pre);
    s_h[s][j] = pre > 0.f ? pre : 0.f;
  }
  __syncthreads();
  if (j < ns) {  // thread j now stands for sample j of the chunk
    float l = w[R_B2];
    for (int u = 0; u < RH; ++u) l = fmaf(w[R_W2 + u], s_h[j][u], l);
    const float y = Y[order[ebase + j]];
    const float p = 1.0f / (1.0f + expf(-l));
    s_g[j] = (p - y) * inv_nb;
    s_l[j] = fmaxf(l, 0.f) - y * l + log1pf(expf(-fabsf(l)));
  }
  __syncthreads();
  float gW[RZ];
#pragma unroll
  for (int k = 0; k < RZ; ++k) gW[k] = 0.f;
  float gb1 = 0.f, gw2 = 0.f;
  for (int s = 0; s < ns; ++s) {
    const float g = s_g[s], h = s_h[s][j];
    gw2 = fmaf(g, h, gw2);
    const float dh = h > 0.f ? g * w2j : 0.f;
    gb1 += dh;
#pragma unroll
    for (int k = 0; k < RZ; ++k) gW[k] = fmaf(s_z[s][k], dh, gW[k]);
  }
  float* P = part + (size_t)blockIdx.x * RT_NPART;
#pragma unroll
  for (int k = 0; k < RZ; ++k) P[k * RH + j] = gW[k];
  P[R_B1 + j] = gb1;
  P[R_W2 + j] = gw2;
  if (j == 0) {
    float gs = 0.f, ls = 0.f;
    for (int s = 0; s < ns; ++s) {
      gs += s_g[s];
      ls += s_l[s];
    }
    P[R_B2] = gs;
    P[RPARAM] = ls;
  }
}

// grad[p] = sum over blocks (in block order); loss[epoch] += loss sum * loss_scale.
__global__ void k_reuse_reduce(const float* __restrict__ part, int nblk, float* __restrict__ grad,
                               float* __restrict__ loss, const uint32_t* __restrict__ ctl, float loss_scale) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < RT_NPART; p += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)b * RT_NPART + p];
    if (p < RPARAM)
      grad[p] = s;
    else
      loss[ctl[1]] += s * loss_scale;
  }
}

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__global__ void k_reuse_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                             float* __restrict__ w, const float* __restrict__ grad, const uint32_t* __restrict__ ctl,
                             float lr) {
  const float t = (float)(ctl[0] + 1u);
  const float bc1 = 1.0f - powf(0.9f, t), bc2 = 1.0f - powf(0.999f, t);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < RPARAM; p += gridDim.x * blockDim.x) {
    const float g = grad[p];
    const float mm = 0.9f * m[p] + 0.1f * g;
    const float vv = 0.999f * v[p] + 0.001f * g * g;
    m[p] = mm;
    v[p] = vv;
    const float th = theta[p] - lr * (mm / bc1) / (sqrtf(vv / bc2) + 1e-8f);
    theta[p] = th;
    w[p] = bf16_round(th);
  }
}

__global__ void k_reuse_tick(uint32_t* ctl, int which) {
  if (threadIdx.x == 0 && blockIdx.x == 0) ctl[which] += 1u;
}

__global__ void k_reuse_round(const float* __restrict__ theta, float* __restrict__ w) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < RPARAM; p += gridDim.x * blockDim.x)
    w[p] = bf16_round(theta[p]);
}

void launch_reuse_round(const float* theta, float* w, cudaStream_t s) { k_reuse_round<<<3, 1024, 0, s>>>(theta, w); }

int reuse_blocks(uint32_t nb) { return (int)((nb + RT_CHUNK - 1) / RT_CHUNK); }

// One mini-batch: samples order[epoch * n_total + b0 + i], i < nb.  With
// lr <= 0 only the gradient (and the loss) is formed.
void launch_reuse_batch(const ReuseTrain& T, uint32_t n_total, uint32_t b0, uint32_t nb, float lr, float loss_scale,
                        cudaStream_t s) {
  const int nblk = reuse_blocks(nb);
  k_reuse_fwdbwd<<<nblk, RH, 0, s>>>(T.Z, T.Y, T.order, T.ctl, n_total, b0, nb, 1.0f / (float)nb, T.w, T.part);
  k_reuse_reduce<<<(RT_NPART + 255) / 256, 256, 0, s>>>(T.part, nblk, T.grad, T.loss, T.ctl, loss_scale);
  if (lr > 0.f) {
    k_reuse_adam<<<3, 1024, 0, s>>>(T.theta, T.m, T.v, T.w, T.grad, T.ctl, lr);
    k_reuse_tick<<<1, 32, 0, s>>>(T.ctl, 0);
  }
}

void launch_reuse_epoch_end(const ReuseTrain& T, cudaStream_t s) { k_reuse_tick<<<1, 32, 0, s>>>(T.ctl, 1); }

}  // namespace gsc
