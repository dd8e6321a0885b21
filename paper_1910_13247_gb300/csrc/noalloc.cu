// mfx_dot_noalloc: the FP64-accumulated dot product of mfx_dot for callers that cannot
// allocate device memory.  Some callers may not call cudaMalloc at all: a plug-in whose host
// application owns every device byte and hands out only the buffers it works on, host code
// that lives inside another runtime's memory budget, where every device byte must come from
// that runtime's pool, and loops that must not block on the allocator (cudaMalloc may
// synchronise the device).  mfx_dot keeps its reduction partials in memory owned by an operator; this
// variant keeps them in a fixed array compiled into the library instead, so it needs neither
// an operator nor an allocation.
//
// The array (kPartials doubles plus a counter, about 8 KB) lives in every GPU that loads the
// library until the process exits.  Its device address is looked up once per device, on the
// first call made with that device current (cudaGetSymbolAddress).  All calls share the array and it keeps the last
// call's contents: each call clears the counter itself, and calls that overlap on the GPU
// (different streams, or different host threads) race on the array and give wrong results.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "mfx_internal.h"

namespace mfx {
namespace {

constexpr int kThreads = 256;
constexpr int kPartials = 1024;  // maximum number of CTAs, one FP64 partial each
constexpr size_t kScratchBytes = kPartials * sizeof(double) + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct DeviceScratch {
  double* partials = nullptr;
  unsigned int* counter = nullptr;
};

template <typename Real>
__global__ void dot_noalloc_kernel(int64_t n, const Real* __restrict__ a, const Real* __restrict__ b,
                                   double* result, double* partials, unsigned int* counter) {
  __shared__ double warp_sums[kThreads / 32];
  __shared__ bool last;
  double v = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v += (double)a[i] * (double)b[i];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) warp_sums[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < kThreads / 32 ? warp_sums[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = v;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  // the last CTA sums the partials: strided loads from L2 by all its threads, then a block sum
  __threadfence();
  double s = 0.0;
  for (unsigned int k = threadIdx.x; k < gridDim.x; k += blockDim.x) s += __ldcg(partials + k);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) warp_sums[warp] = s;  // its first use ended before the barrier that published `last`
  __syncthreads();
  if (warp == 0) {
    s = lane < kThreads / 32 ? warp_sums[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) {
      *result = s;
      *counter = 0u;
    }
  }
}

mfx_status device_scratch(DeviceScratch* out) {
  static std::mutex lock;
  static DeviceScratch table[64];
  int dev = 0;
  MFX_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(MFX_EUNSUPPORTED, "mfx_dot_noalloc: device index above 63");
  std::lock_guard<std::mutex> g(lock);
  if (!table[dev].partials) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    table[dev].partials = static_cast<double*>(p);
    table[dev].counter = reinterpret_cast<unsigned int*>(static_cast<unsigned char*>(p) + kPartials * sizeof(double));
  }
  *out = table[dev];
  return MFX_OK;
}

}  // namespace
}  // namespace mfx

using namespace mfx;

extern "C" mfx_status mfx_dot_noalloc(mfx_prec prec, int64_t n, const void* a, const void* b, double* result,
                                      mfx_stream stream) {
  if (!a || !b || !result || (prec != MFX_F64 && prec != MFX_F32))
    return set_error(MFX_EINVAL, "mfx_dot_noalloc: null pointer or unknown precision");
  if (n < 0 || n > MFX_NOALLOC_MAX_N)
    return set_error(MFX_EINVAL, "mfx_dot_noalloc: n must be in 0..MFX_NOALLOC_MAX_N (2^31 - 1)");
  DeviceScratch sc;
  mfx_status st = device_scratch(&sc);
  if (st != MFX_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = std::min(reduction_blocks(n), kPartials);
  MFX_CUDA_TRY(cudaMemsetAsync(sc.counter, 0, sizeof(unsigned int), s));
  if (prec == MFX_F64)
    dot_noalloc_kernel<double><<<grid, kThreads, 0, s>>>(n, (const double*)a, (const double*)b, result, sc.partials,
                                                          sc.counter);
  else
    dot_noalloc_kernel<float><<<grid, kThreads, 0, s>>>(n, (const float*)a, (const float*)b, result, sc.partials,
                                                         sc.counter);
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}
