// TMA and mbarrier building blocks of the FP32 brick-row kernel (vmult_brick_tma2.cuh).
//
// The n^2 lattice rows of a batch are moved by the Tensor Memory Accelerator: one 1D tensor copy per
// row into shared memory (tracked by an mbarrier, issued one batch ahead into a second buffer) and
// one 1D tensor reduce-add per row from shared memory into dst.  Rows start at arbitrary DoF
// offsets, so each copy starts at the 16-byte boundary below the row and the row sits at offset
// (start mod 4) inside its tile row.  Every wait on an mbarrier is bounded (about one second of
// clock); a timeout sets an error word, drains the CTA's outstanding copies and ends the CTA.
#pragma once

#include <cuda.h>

#include "vmult_brick.cuh"

namespace mfx {

template <int N, int CB>
struct TmaShape {
  static constexpr int K = N - 1;
  static constexpr int ROWS = N * N;
  static constexpr int WMAX = CB * K + 1;
  static constexpr int BOX = (WMAX + 3 + 3) / 4 * 4;  // row shifted by up to 3 points, 16-byte multiple
  static constexpr int PITCH = (BOX + 31) / 32 * 32;  // 128-byte aligned tile rows
  static constexpr int TILE = ROWS * PITCH;
  static_assert(BOX <= 256, "TMA box dimension");
};

template <int N>
struct TmaArgs {
  CUtensorMap tsrc;  // 1D float map of src (loads)
  CUtensorMap tdst;  // 1D float map of dst (reduce-add)
  const float* metric;
  int nx, ny, nz, nchunk;
  int Mx, My, Mz;
  int n_batches;
  int* err;               // set to 1 if a bounded wait ran out
  const int32_t* skip;
  uint32_t dmask;         // Dirichlet faces
  int step_chunk, step_y, step_z;  // the grid size as (chunk, y, z) steps of batch positions
  // plain pointers and length of src and dst (kernels that move tile rows by untiled bulk copies)
  const float* src;
  float* dst;
  int64_t n;
  // box cells (the BOXM kernel variants): w_q / w_0 of the 1D Gauss weights; the metric along a line is
  // these ratios times the line's first point's diagonal
  float wr[N];
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// Bounded wait for the phase with the given parity; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const long long start = clock64();
  for (;;) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - start > (1ll << 31)) return false;
  }
}
__device__ __forceinline__ void tma_load_1d(float* dst, const CUtensorMap* map, int x, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.1d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2}], [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_reduce_add_1d(const CUtensorMap* map, int x, const float* src) {
  asm volatile("cp.reduce.async.bulk.tensor.1d.global.shared::cta.add.tile.bulk_group [%0, {%1}], [%2];\n" ::"l"(map),
               "r"(x), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(PENDING) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// Hint to the TMA engine: bring `bytes` (a multiple of 16, 16-byte aligned, inside one allocation) of
// global memory into L2; nothing waits for it.
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

}  // namespace mfx
