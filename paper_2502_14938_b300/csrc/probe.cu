// gsc_debug_pipe_rates: measured issue rates of the arithmetic units the
// blend leans on, for its roofline.  Each kernel runs independent dependency
// chains of one instruction kind (8 per thread, long enough to hide latency)
// on 8 blocks of 256 threads per SM and stores one float per thread, so the
// timed rate is the unit's throughput: exp2 results per second (the special
// function unit), FP32 FMA lane operations per second (scalar FFMA), and
// lane operations per second of the packed FP32x2 FMA (each FFMA2 counts
// two).  Values do not matter; the chains saturate to inf or a fixed point.
#include <cuda_runtime.h>

#include "gsc.h"
#include "gsc_debug.h"

namespace gsc {
namespace {

constexpr int PROBE_CHAINS = 8, PROBE_ITERS = 4096, PROBE_THREADS = 256;

__global__ void k_probe_ex2(float* out, float seed) {
  float x[PROBE_CHAINS];
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = seed * (float)(threadIdx.x + i) * 1e-9f - 1.f;
  for (int it = 0; it < PROBE_ITERS; ++it)
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(x[i]));
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_probe_ffma(float* out, float seed) {
  float x[PROBE_CHAINS];
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = (float)(threadIdx.x + i);
  for (int it = 0; it < PROBE_ITERS; ++it)
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[i]) : "f"(0.999f), "f"(seed));
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_probe_ffma2(float* out, float seed) {
  unsigned long long x[PROBE_CHAINS], a, b;
  asm("mov.b64 %0, {%1, %1};" : "=l"(a) : "f"(0.999f));
  asm("mov.b64 %0, {%1, %1};" : "=l"(b) : "f"(seed));
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; ++i)
    asm("mov.b64 %0, {%1, %2};" : "=l"(x[i]) : "f"((float)i), "f"((float)threadIdx.x));
  for (int it = 0; it < PROBE_ITERS; ++it)
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[i]) : "l"(a), "l"(b));
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; ++i) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[i]));
    s += lo + hi;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Median of 5 timed launches (after 2 untimed), in seconds.
template <typename K>
int time_probe(K kern, float* out, int blocks, cudaStream_t s, double* sec) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return GSC_ERR_CUDA;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return GSC_ERR_CUDA;
  }
  float t[5];
  for (int r = 0; r < 7; ++r) {
    cudaEventRecord(a, s);
    kern<<<blocks, PROBE_THREADS, 0, s>>>(out, 0.5f);
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    if (r >= 2) cudaEventElapsedTime(&t[r - 2], a, b);
  }
  const cudaError_t e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return GSC_ERR_CUDA;
  for (int i = 0; i < 5; ++i)
    for (int j = i + 1; j < 5; ++j)
      if (t[j] < t[i]) {
        const float x = t[i];
        t[i] = t[j];
        t[j] = x;
      }
  *sec = t[2] * 1e-3;
  return GSC_OK;
}

}  // namespace
}  // namespace gsc

int gsc_debug_pipe_rates(double* rates) {
  using namespace gsc;
  if (!rates) return GSC_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return GSC_ERR_CUDA;
  const int blocks = sms * 8;
  float* out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * PROBE_THREADS * sizeof(float)) != cudaSuccess) return GSC_ERR_OOM;
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFree(out);
    return GSC_ERR_CUDA;
  }
  const double ops = (double)blocks * PROBE_THREADS * PROBE_CHAINS * PROBE_ITERS;
  double t0 = 0, t1 = 0, t2 = 0;
  int r = time_probe(k_probe_ex2, out, blocks, s, &t0);
  if (!r) r = time_probe(k_probe_ffma, out, blocks, s, &t1);
  if (!r) r = time_probe(k_probe_ffma2, out, blocks, s, &t2);
  cudaStreamDestroy(s);
  cudaFree(out);
  if (r) return r;
  rates[0] = ops / t0;
  rates[1] = ops / t1;
  rates[2] = 2.0 * ops / t2;
  return GSC_OK;
}
