// Self-test of failure detection without a fault: one CTA waits on a shared-memory mbarrier at which
// nothing ever arrives, through the bounded wait of the TMA kernels (mbar_wait: about 2^31 SM clocks,
// about one second at 2 GHz).  The wait runs out, the kernel sets the operator's error word and
// returns, the context stays usable, and mfx_device_check reports MFX_ETIMEOUT.
#include <cuda_runtime.h>

#include "mfx_internal.h"
#include "vmult_brick_tma.cuh"

namespace mfx {
namespace {

__global__ void bounded_wait_selftest_kernel(int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);  // one arrival expected; none is ever made
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0)) atomicExch(err, 1);
}

}  // namespace
}  // namespace mfx

using namespace mfx;

extern "C" mfx_status mfx_selftest_bounded_wait(const mfx_op* op, mfx_stream stream) {
  if (!op || !op->d_err) return set_error(MFX_EINVAL, "mfx_selftest_bounded_wait: null operator");
  bounded_wait_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(op->d_err);
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}
