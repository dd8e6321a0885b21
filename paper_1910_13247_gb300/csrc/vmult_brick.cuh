// Matrix-free Q_k Laplacian on structured meshes: "brick-row" kernel.
//
// A batch is CB consecutive cells along x in one row (cy, cz).  Per batch:
//  0. the batch's DoFs, (CB k + 1) x n x n lattice points in n^2 contiguous
//     rows of the global vector, are copied into a row-major shared-memory
//     tile with 4/8-byte asynchronous copies (cp.async), one batch ahead
//     for FP32 (double-buffered); Dirichlet points are stored as 0;
//  1. forward 1D contractions (tensor-product evaluation, Sec. 3.6):
//     S_z (reading z-lines straight from the tile), S_y, S_x (values at the
//     Gauss points), then D_x (registers), D_y, D_z (reference gradient);
//  2. h = G_q grad at every Gauss point, G prefetched into registers at the
//     start of the batch (six entries per point stored as [batch][6][q][CB],
//     so that the loads of a warp are coalesced);
//  3. transposed contractions D^T, summed over the three components, then
//     S_x^T, S_y^T, and S_z^T writing straight into a row-major output
//     tile (nodes shared by neighbouring cells are summed in two passes);
//  4. the tile is added to dst with coalesced atomic adds (Dirichlet rows
//     get dst = src; dst is zeroed before the launch).
// Every 1D contraction is done by a thread owning one line of one cell;
// lanes run over cells fastest, and the cube paddings (NP, P2, CELL) and the
// tile skew/pitch were chosen so that the line accesses of a warp are free
// of shared-memory bank conflicts (FP32 words; the tile phases of even n
// keep a 1.5-way conflict).
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

template <int N, typename Real, int CB>
__global__ void __launch_bounds__(BrickShape<N, CB, Real>::THREADS,
                                  (sizeof(Real) == 4 ? (1024 / BrickShape<N, CB, Real>::THREADS > 0
                                                            ? 1024 / BrickShape<N, CB, Real>::THREADS : 1) : 1))
    brick_vmult_kernel(const __grid_constant__ BrickArgs<N, Real> a, const Real* __restrict__ src,
                       Real* __restrict__ dst) {
  using Sh = BrickShape<N, CB, Real>;
  constexpr int K = Sh::K, NP = Sh::NP, P2 = Sh::P2, CELL = Sh::CELL, N3 = N * N * N;
  constexpr int PITCH = Sh::PITCH, SKEW = Sh::SKEW, WMAX = Sh::WMAX;
  constexpr bool PREFETCH = 6 * N * (int)sizeof(Real) / 4 <= 32;
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* tiles = reinterpret_cast<Real*>(smem_raw);
  Real* A = tiles + Sh::NBUF * Sh::TILE;
  Real* B = A + Sh::CUBES;
  Real* C = B + Sh::CUBES;

  const int t = threadIdx.x;
  const int c = t % CB;
  const int r = t / CB;
  const int f = r % N, s = r / N;
  const bool line_ok = t < Sh::LINES;
  // line bases in the cubes
  const int xa2 = Sh::XSWAP ? s : f, xa3 = Sh::XSWAP ? f : s;
  const int xbase = c * CELL + xa3 * P2 + xa2 * NP;  // x-line (a2, a3), stride 1
  const int ybase = c * CELL + s * P2 + f;          // y-line (a1 = f, a3 = s), stride NP
  const int zbase = c * CELL + s * NP + f;          // z-line (a1 = f, a2 = s), stride P2
  // z-line (a1 = f, a2 = s) in the tile: point x = c K + f of rows a3 N + s
  const int zx = c * K + f;
  const int ztile = s * PITCH + zx + (zx / K) * SKEW;  // + a3 * N * PITCH
  const int n_batches = (int)a.n_batches;

  // issue the asynchronous copies of batch bb into tile buffer `buf` (Dirichlet points set to 0);
  // warp w copies tile rows w, w + NWARPS, ...; lanes walk the points of the row
  constexpr int NWARPS = Sh::THREADS / 32, XITERS = (WMAX + 31) / 32;
  const int warp = t >> 5, lane = t & 31;
  auto load_tile = [&](int bb, Real* buf) {
    const BatchInfo bi = batch_info<CB, K>(a, bb);
    for (int row = warp; row < N * N; row += NWARPS) {
      const int a2 = row % N, a3 = row / N;
      const int rflags = (a2 == 0 ? 1 : 0) | (a2 == K ? 2 : 0) | (a3 == 0 ? 4 : 0) | (a3 == K ? 8 : 0);
      const bool rbnd = (rflags & bi.eflags) != 0;
      const Real* g = src + bi.gbase + a.Mx * (a2 + a.My * a3);
      Real* p = buf + row * PITCH;
#pragma unroll
      for (int j = 0; j < XITERS; ++j) {
        const int x = lane + 32 * j;
        if (x < bi.Wm) {
          const bool bnd = rbnd || (x == 0 && bi.xlo) || (x == bi.Wm - 1 && bi.xhi);
          Real* q = p + x + (x / K) * SKEW;
          if (bnd)
            *q = Real(0);
          else
            cp_async(q, g + x);
        }
      }
    }
    cp_async_commit();
  };

  int buf = 0;
  if (Sh::NBUF == 2 && (int)blockIdx.x < n_batches) load_tile(blockIdx.x, tiles);

  for (int b = blockIdx.x; b < n_batches; b += gridDim.x) {
    const BatchInfo bi = batch_info<CB, K>(a, b);
    const int m = bi.m;
    const bool act = line_ok && c < m;
    const Real* Gb = a.metric + (int64_t)b * (6 * N3 * CB) + (xa2 * N + xa3 * N * N) * CB + c;
    Real* T = tiles + buf * Sh::TILE;

    if constexpr (Sh::NBUF == 2) {
      // copies of the next batch go into the other buffer; this batch's copies were issued earlier
      if (b + (int)gridDim.x < n_batches) load_tile(b + gridDim.x, tiles + (buf ^ 1) * Sh::TILE);
      else cp_async_commit();
      cp_async_wait<1>();
    } else {
      load_tile(b, T);
      cp_async_wait<0>();
    }
    // metric of this thread's x-line, consumed four phases later
    Real G[PREFETCH ? 6 : 1][N];
    if (PREFETCH && act) {
#pragma unroll
      for (int e = 0; e < 6; ++e)
#pragma unroll
        for (int q = 0; q < N; ++q) G[e][q] = __ldg(Gb + (e * N3 + q) * CB);
    }
    __syncthreads();
    // 1) S along z: z-lines from the tile into cube A
    if (act) {
      Real v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = T[ztile + j * N * PITCH];
      contract<N, Real, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[zbase + j * P2] = o[j];
    }
    __syncthreads();
    // 2) S along y
    if (act) {
      Real v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[ybase + j * NP];
      contract<N, Real, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[ybase + j * NP] = o[j];
    }
    __syncthreads();
    // 3) S along x -> values at Gauss points; D along x kept in registers
    Real g1[N];
    if (act) {
      Real v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[xbase + j];
      contract<N, Real, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[xbase + j] = o[j];
      contract<N, Real, MAT_D>(o, g1);
    }
    __syncthreads();
    // 4) D along y -> B, D along z -> C
    if (act) {
      Real v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[ybase + j * NP];
      contract<N, Real, MAT_D>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) B[ybase + j * NP] = o[j];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[zbase + j * P2];
      contract<N, Real, MAT_D>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) C[zbase + j * P2] = o[j];
    }
    __syncthreads();
    // 5) quadrature-point metric on the x-line; D_x^T in registers
    Real t1[N];
    if (act) {
      Real h1[N];
#pragma unroll
      for (int q = 0; q < N; ++q) {
        Real G00, G01, G02, G11, G12, G22;
        if constexpr (PREFETCH) {
          G00 = G[0][q]; G01 = G[1][q]; G02 = G[2][q]; G11 = G[3][q]; G12 = G[4][q]; G22 = G[5][q];
        } else {
          G00 = __ldg(Gb + (0 * N3 + q) * CB); G01 = __ldg(Gb + (1 * N3 + q) * CB);
          G02 = __ldg(Gb + (2 * N3 + q) * CB); G11 = __ldg(Gb + (3 * N3 + q) * CB);
          G12 = __ldg(Gb + (4 * N3 + q) * CB); G22 = __ldg(Gb + (5 * N3 + q) * CB);
        }
        const Real u1 = g1[q], u2 = B[xbase + q], u3 = C[xbase + q];
        h1[q] = G00 * u1 + G01 * u2 + G02 * u3;
        B[xbase + q] = G01 * u1 + G11 * u2 + G12 * u3;
        C[xbase + q] = G02 * u1 + G12 * u2 + G22 * u3;
      }
      contract_t<N, Real, MAT_D>(h1, t1);
    }
    __syncthreads();
    // 6) D_y^T on B, D_z^T on C
    if (act) {
      Real v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = B[ybase + j * NP];
      contract_t<N, Real, MAT_D>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) B[ybase + j * NP] = o[j];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = C[zbase + j * P2];
      contract_t<N, Real, MAT_D>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) C[zbase + j * P2] = o[j];
    }
    __syncthreads();
    // 7) sum of the three components, S_x^T -> A
    if (act) {
      Real v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = t1[j] + B[xbase + j] + C[xbase + j];
      contract_t<N, Real, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[xbase + j] = o[j];
    }
    __syncthreads();
    // 8) S_y^T
    if (act) {
      Real v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[ybase + j * NP];
      contract_t<N, Real, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[ybase + j * NP] = o[j];
    }
    __syncthreads();
    // 9) S_z^T into the output tile (aliases this batch's input tile, consumed in step 1):
    //    nodes with a1 < K first, then the a1 = K nodes add to the next cell's a1 = 0 node
    Real o9[N];
    if (act) {
      Real v[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[zbase + j * P2];
      contract_t<N, Real, MAT_S>(v, o9);
      if (f < K) {
#pragma unroll
        for (int j = 0; j < N; ++j) T[ztile + j * N * PITCH] = o9[j];
      }
    }
    __syncthreads();
    if (act && f == K) {
      if (c < m - 1) {
#pragma unroll
        for (int j = 0; j < N; ++j) T[ztile + j * N * PITCH] += o9[j];
      } else {
#pragma unroll
        for (int j = 0; j < N; ++j) T[ztile + j * N * PITCH] = o9[j];
      }
    }
    __syncthreads();
    // 10) scatter: coalesced atomic adds, warp per tile row; constrained rows copy src
    for (int row = warp; row < N * N; row += NWARPS) {
      const int a2 = row % N, a3 = row / N;
      const int rflags = (a2 == 0 ? 1 : 0) | (a2 == K ? 2 : 0) | (a3 == 0 ? 4 : 0) | (a3 == K ? 8 : 0);
      const bool rbnd = (rflags & bi.eflags) != 0;
      const int g = bi.gbase + a.Mx * (a2 + a.My * a3);
      const Real* p = T + row * PITCH;
#pragma unroll
      for (int j = 0; j < XITERS; ++j) {
        const int x = lane + 32 * j;
        if (x < bi.Wm) {
          const bool bnd = rbnd || (x == 0 && bi.xlo) || (x == bi.Wm - 1 && bi.xhi);
          if (bnd)
            dst[g + x] = __ldg(src + g + x);
          else
            red_add(dst + g + x, p[x + (x / K) * SKEW]);
        }
      }
    }
    __syncthreads();
    buf ^= (Sh::NBUF - 1);
  }
  if constexpr (Sh::NBUF == 2) cp_async_wait<0>();
}

}  // namespace mfx
