// gsc_scan_u32_noalloc: the decoupled look-back exclusive scan for callers
// that may not allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a scan:
// a frame loop that runs under a real-time budget (an allocation can
// synchronise the device and stall the frame), or a host application that
// owns every device allocation through its own pool and hands plug-ins only
// the buffers they work on.  This entry point takes the caller's device
// input and output and keeps its own working memory (the look-back words of
// every 4096-element tile plus three control words) in one file-scope device
// array of fixed size, so a call allocates nothing.
//
// The array costs 4100 x 8 = 32,800 bytes on every GPU that loads the
// library, held until the process exits.  Host code cannot use the array's
// name as a device address, so every call looks the address up with
// cudaGetSymbolAddress for the device (and context) current at the call and
// passes it to the kernels; nothing is cached across calls, so a reset
// device or another context on the same device gets its own array's
// address.  Every call shares the
// array: the call resets the tile counter and error word and advances an
// epoch, so look-back words left by earlier calls are never mistaken for
// this call's; two calls whose kernels overlap on the GPU (other host
// threads, other streams) race on the array and must be serialised by the
// caller.
#include <cuda_runtime.h>

#include "gsc.h"
#include "gsc_internal.cuh"

namespace gsc {
namespace {

constexpr int NA_NT = 256;
constexpr int NA_IPT = 16;
constexpr uint32_t NA_TILE = NA_NT * NA_IPT;  // 4096 elements per tile
constexpr uint32_t NA_MAX_TILES = GSC_NOALLOC_SCAN_MAX_N / NA_TILE;
constexpr uint32_t NA_WORDS = NA_MAX_TILES + 4;  // look-back words + control words
constexpr uint32_t NA_CTRL = NA_MAX_TILES;       // [ctrl] tile counter, [ctrl+1] epoch, [ctrl+2] error bits
constexpr uint32_t NA_ERR_SUM = 16u;             // the running sum reached 2^30
constexpr uint32_t NA_SPIN = 1u << 20;

static __device__ __align__(256) unsigned long long g_noalloc_scan_scratch[NA_WORDS];

__global__ void k_noalloc_begin(unsigned long long* scratch) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  *reinterpret_cast<uint32_t*>(scratch + NA_CTRL) = 0;  // tile counter
  uint32_t* epoch = reinterpret_cast<uint32_t*>(scratch + NA_CTRL + 1);
  *epoch = *epoch + 1u;
  uint32_t* err = reinterpret_cast<uint32_t*>(scratch + NA_CTRL + 2);
  *err = 0;
}

// `in` may equal `out` (in place: a tile reads all its inputs before it
// writes), so neither pointer is declared __restrict__.
__global__ void __launch_bounds__(NA_NT) k_noalloc_scan(const uint32_t* in, uint32_t* out, uint32_t n,
                                                        uint32_t* total_out, unsigned long long* scratch) {
  __shared__ uint32_t s_warp[NA_NT / 32 + 1];
  __shared__ unsigned long long s_sum64[NA_NT / 32];
  __shared__ uint32_t s_base;
  __shared__ uint32_t s_tile;
  uint32_t* ctr = reinterpret_cast<uint32_t*>(scratch + NA_CTRL);
  const uint32_t epoch = *reinterpret_cast<volatile uint32_t*>(scratch + NA_CTRL + 1);
  uint32_t* err = reinterpret_cast<uint32_t*>(scratch + NA_CTRL + 2);
  const uint32_t ntiles = (n + NA_TILE - 1) / NA_TILE;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(ctr, 1u);
    __syncthreads();
    const uint32_t t = s_tile;
    if (t >= ntiles) break;
    const uint32_t i0 = t * NA_TILE + threadIdx.x * NA_IPT;
    uint32_t v[NA_IPT];
    unsigned long long sum64 = 0;
#pragma unroll
    for (int u = 0; u < NA_IPT; ++u) {
      const uint32_t i = i0 + u;
      v[u] = i < n ? in[i] : 0u;
      sum64 += v[u];
    }
    // exact tile total in 64 bits to detect sums the 30-bit look-back words cannot hold
    unsigned long long w64 = sum64;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w64 += __shfl_xor_sync(0xffffffffu, w64, o);
    if ((threadIdx.x & 31u) == 0) s_sum64[threadIdx.x >> 5] = w64;
    const uint32_t sum = sum64 < (1ull << 30) ? (uint32_t)sum64 : (1u << 30);
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan<NA_NT>(sum, s_warp, &tot);
    if (threadIdx.x == 0) {
      unsigned long long tot64 = 0;
      for (int w = 0; w < NA_NT / 32; ++w) tot64 += s_sum64[w];
      if (tot64 >= (1ull << 30)) atomicOr(err, NA_ERR_SUM);
      unsigned long long* wd = scratch + t;
      uint32_t pre = 0;
      if (t == 0) {
        st_relaxed_u64(wd, lb_pack(epoch, 2u, tot));
      } else {
        st_relaxed_u64(wd, lb_pack(epoch, 1u, tot));
        pre = lb_exclusive(scratch, 1, t, epoch, NA_SPIN, err);
        st_relaxed_u64(wd, lb_pack(epoch, 2u, pre + tot));
      }
      if ((unsigned long long)pre + tot64 >= (1ull << 30)) atomicOr(err, NA_ERR_SUM);
      s_base = pre;
      if (t == ntiles - 1 && total_out) *total_out = pre + tot;
    }
    __syncthreads();
    uint32_t run = s_base + ex;
#pragma unroll
    for (int u = 0; u < NA_IPT; ++u) {
      const uint32_t i = i0 + u;
      if (i < n) out[i] = run;
      run += v[u];
    }
    __syncthreads();
  }
}

}  // namespace
}  // namespace gsc

extern "C" int gsc_scan_u32_noalloc(const uint32_t* d_in, uint32_t* d_out, uint64_t n, uint32_t* d_total,
                                    void* cuda_stream) {
  using namespace gsc;
  if (n > GSC_NOALLOC_SCAN_MAX_N) return GSC_ERR_INVALID_ARG;
  if (n > 0 && (!d_in || !d_out)) return GSC_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // the call ends by reading the error word back and synchronising the
  // stream, neither of which a stream under capture allows
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return GSC_ERR_CUDA;
  if (cap != cudaStreamCaptureStatusNone) return GSC_ERR_INVALID_ARG;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GSC_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
    return GSC_ERR_CUDA;
  // the device address of this context's copy of the array (the array's
  // name in host code is only a stand-in for it)
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scan_scratch) != cudaSuccess || !p) return GSC_ERR_CUDA;
  unsigned long long* scratch = static_cast<unsigned long long*>(p);
  if (n == 0) {
    if (d_total && cudaMemsetAsync(d_total, 0, sizeof(uint32_t), s) != cudaSuccess) return GSC_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? GSC_OK : GSC_ERR_CUDA;
  }
  k_noalloc_begin<<<1, 32, 0, s>>>(scratch);
  const uint32_t ntiles = (uint32_t)((n + NA_TILE - 1) / NA_TILE);
  const uint32_t grid = ntiles < (uint32_t)(2 * nsm) ? ntiles : (uint32_t)(2 * nsm);
  k_noalloc_scan<<<grid, NA_NT, 0, s>>>(d_in, d_out, (uint32_t)n, d_total, scratch);
  if (cudaGetLastError() != cudaSuccess) return GSC_ERR_CUDA;
  uint32_t err = 0;
  const void* err_addr = reinterpret_cast<const char*>(scratch + NA_CTRL + 2);
  if (cudaMemcpyAsync(&err, err_addr, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GSC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return GSC_ERR_CUDA;
  if (err & NA_ERR_SUM) return GSC_ERR_INVALID_ARG;
  if (err & ERR_TIMEOUT) return GSC_ERR_TIMEOUT;
  return GSC_OK;
}
