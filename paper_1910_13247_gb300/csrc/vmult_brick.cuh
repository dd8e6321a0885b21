// Structured meshes, "brick rows": shared definitions of the batched kernels.
//
// A batch is CB consecutive cells along x in one row (cy, cz); its DoFs are the (CB k + 1) x n x n
// lattice points in n^2 contiguous rows of the global vector.  This header holds what the FP32
// paired kernel (vmult_brick_tma2.cuh) and the FP64 double-float kernel (vmult_brick_df.cuh) share:
// the batch sizes compiled per degree, the shared-memory shapes (cube paddings NP, P2, CELL and the
// tile pitch/skew, chosen so that the line accesses of a warp are free of bank conflicts), the
// per-batch Dirichlet flags and positions, and the cp.async helpers.  Every 1D contraction is done
// by a thread owning one line of one cell (or of a pair of cells); lanes run over cells fastest, so
// the metric, stored per batch as [batch][6][q][CB], is loaded coalesced.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vmult.cuh"

namespace mfx {

// cells per batch for each n (= k + 1)
template <int N> struct BrickCB {
  static constexpr int value = N == 2 ? 32 : (N <= 7 ? 16 : 8);  // default
  static constexpr int ALT = (N == 4 || N == 5) ? 8 : N == 3 ? 32 : 0;  // second compiled choice (0: none)
};

template <int N, int CB, typename Real>
struct BrickShape {
  static constexpr int K = N - 1;
  static constexpr int LINES = CB * N * N;
  static constexpr int THREADS = (LINES + 31) / 32 * 32;
  static constexpr bool XSWAP = (N % 2) == 0;
  // conflict-free cube paddings
  static constexpr int NP = N;
  static constexpr int P2 = N == 2 ? (CB == 16 ? 5 : 4) : N == 3 ? 9 : N == 4 ? 17 : N == 5 ? 25 : N == 6 ? 37
                          : N == 7 ? 49 : N == 8 ? 65 : 81;
  static constexpr int CELL = N == 2 ? (CB == 16 ? 10 : 9) : N == 3 ? (CB == 16 ? 30 : 27)
                            : N == 4 ? (CB == 8 ? 68 : 70) : N == 5 ? (CB == 8 ? 132 : CB == 32 ? 125 : 126)
                            : N == 6 ? 222 : N == 7 ? 346 : N == 8 ? (CB == 4 ? 520 : 524) : (CB == 4 ? 744 : 732);
  static constexpr int CUBES = CB * CELL;  // elements per cube array
  // row-major tile: point x of row r at r * PITCH + x + (x / K) * SKEW
  static constexpr int WMAX = CB * K + 1;
  static constexpr bool F32 = sizeof(Real) == 4;
  static constexpr int SKEW = !F32 ? 0 : N == 4 ? 3 : N == 5 ? 2 : N == 6 ? 1 : N == 8 ? 5 : 0;
  static constexpr int PITCH_MIN = WMAX + (WMAX - 1) / K * SKEW;
  static constexpr int PITCH_TABLE = N <= 3 ? 33 : 97;  // conflict-free pitches found for the default CB
  static constexpr int PITCH = !F32 ? (WMAX | 1) : (PITCH_TABLE >= PITCH_MIN ? PITCH_TABLE : (PITCH_MIN | 1));
  static_assert(PITCH >= PITCH_MIN, "tile pitch too small");
  static constexpr int TILE = N * N * PITCH;  // elements per tile buffer
  static constexpr int NBUF = F32 ? 2 : 1;    // input tiles (double-buffered for FP32); output aliases
  static constexpr size_t SMEM = (size_t)(NBUF * TILE + 3 * CUBES) * sizeof(Real);
};

template <int N, typename Real>
struct BrickArgs {
  const Real* metric;  // [batch][6][N^3][CB]
  int nx, ny, nz, nchunk;
  int Mx, My, Mz;
  int64_t n_batches;
  const int32_t* skip;
  uint32_t dmask;  // Dirichlet faces
};

template <typename Real>
__device__ __forceinline__ void red_add(Real* p, Real v) {
  atomicAdd(p, v);
}

// Per-batch quantities: valid cells, lattice points per row, first lattice point and the
// Dirichlet tests (row ends in x; the four row edges in y and z as a 4-bit mask).
struct BatchInfo {
  int cx0, m, Wm, gbase, eflags;
  bool xlo, xhi;
};

// Position of batch b: chunk of its row of cells, and the row (cy, cz).
struct BatchPos {
  int chunk, cy, cz;
};

template <typename Args>
__device__ __forceinline__ BatchPos batch_pos(const Args& a, int b) {
  const int row = b / a.nchunk;
  return BatchPos{b - row * a.nchunk, row % a.ny, row / a.ny};
}

// Advance a position by the grid size (a.step_* = the grid size split as chunk, y, z), with carries
// instead of the divisions of batch_pos.
template <typename Args>
__device__ __forceinline__ void batch_advance(BatchPos& p, const Args& a) {
  p.chunk += a.step_chunk;
  const int c1 = p.chunk >= a.nchunk ? 1 : 0;
  p.chunk -= c1 * a.nchunk;
  p.cy += a.step_y + c1;
  const int c2 = p.cy >= a.ny ? 1 : 0;
  p.cy -= c2 * a.ny;
  p.cz += a.step_z + c2;
}

template <int CB, int K, typename Args>
__device__ __forceinline__ BatchInfo batch_info_at(const Args& a, const BatchPos& p) {
  BatchInfo bi;
  const int chunk = p.chunk, cy = p.cy, cz = p.cz;
  bi.cx0 = chunk * CB;
  bi.m = min(CB, a.nx - bi.cx0);
  bi.Wm = bi.m * K + 1;
  bi.gbase = bi.cx0 * K + a.Mx * (cy * K + a.My * (cz * K));
  const uint32_t f = a.dmask;
  bi.xlo = bi.cx0 == 0 && (f & 1u);
  bi.xhi = bi.cx0 + bi.m == a.nx && (f & 2u);
  bi.eflags = (cy == 0 && (f & 4u) ? 1 : 0) | (cy == a.ny - 1 && (f & 8u) ? 2 : 0) | (cz == 0 && (f & 16u) ? 4 : 0) |
              (cz == a.nz - 1 && (f & 32u) ? 8 : 0);
  return bi;
}

template <int CB, int K, typename Args>
__device__ __forceinline__ BatchInfo batch_info(const Args& a, int b) {
  return batch_info_at<CB, K>(a, batch_pos(a, b));
}

template <typename Real>
__device__ __forceinline__ void cp_async(Real* smem, const Real* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (sizeof(Real) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory"); }

}  // namespace mfx
