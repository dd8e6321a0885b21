// Matrix-free Q_k Laplacian on structured meshes: "brick-row" kernel.
//
// A batch is CB consecutive cells along x in one row (cy, cz).  Per batch:
//  0. the DoFs of the batch, (CB k + 1) x n x n lattice points, are read
//     with coalesced row loads and written into per-cell cubes in shared
//     memory (nodes shared by neighbouring cells are stored in both cubes;
//     Dirichlet values read as 0);
//  1. forward 1D contractions (Sec. 3.6, tensor-product evaluation):
//     S_z, S_y, S_x (values at Gauss points), then D_x (registers), D_y, D_z;
//  2. h = G_q grad at every Gauss point (G prefetched from HBM into
//     registers at the start of the batch: 6 values per point, stored
//     interleaved as [batch][6][q][CB] so that loads are coalesced);
//  3. transposed contractions D^T then S^T, summed over the three gradient
//     components;
//  4. the cube results are summed over shared nodes and added to dst with
//     coalesced atomic adds (Dirichlet rows get dst = src).
// Every 1D contraction is done by a thread owning one line of one cell;
// lanes run over cells fastest, and the cube paddings (NP, P2, CELL) were
// chosen so that all line accesses of a warp are free of bank conflicts
// (FP32 words).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vmult.cuh"

namespace mfx {

// cells per batch for each n (= k + 1)
template <int N> struct BrickCB { static constexpr int value = N == 2 ? 32 : (N <= 7 ? 16 : 8); };

template <int N, int CB>
struct BrickShape {
  static constexpr int K = N - 1;
  static constexpr int LINES = CB * N * N;
  static constexpr int THREADS = (LINES + 31) / 32 * 32;
  static constexpr bool XSWAP = (N % 2) == 0;
  // conflict-free paddings (see the layout search in the design notes)
  static constexpr int NP = N;
  static constexpr int P2 = N == 2 ? (CB == 16 ? 5 : 4) : N == 3 ? 9 : N == 4 ? 17 : N == 5 ? 25 : N == 6 ? 37
                          : N == 7 ? 49 : N == 8 ? 65 : 81;
  static constexpr int CELL = N == 2 ? (CB == 16 ? 10 : 9) : N == 3 ? (CB == 16 ? 30 : 27)
                            : N == 4 ? (CB == 8 ? 68 : 70) : N == 5 ? (CB == 8 ? 132 : 126)
                            : N == 6 ? 222 : N == 7 ? 346 : N == 8 ? (CB == 4 ? 520 : 524) : (CB == 4 ? 744 : 732);
  static constexpr int CUBES = CB * CELL;  // elements per cube array
  static constexpr int WMAX = CB * K + 1;  // lattice points per row of a full batch
  static constexpr int TILE = N * N * WMAX;
  static constexpr int TILE_ITERS = (TILE + THREADS - 1) / THREADS;
  // bytes of shared memory before the cubes: the tile descriptor table (2 words per element)
  static constexpr int TABLE_BYTES = (TILE * 8 + 15) / 16 * 16;
};

template <int N, typename Real>
struct BrickArgs {
  const Real* metric;  // [batch][6][N^3][CB]
  int nx, ny, nz, nchunk;
  int Mx, My, Mz;
  int64_t n_batches;
  const int32_t* skip;
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

template <int CB, int K, typename Args>
__device__ __forceinline__ BatchInfo batch_info(const Args& a, int b) {
  BatchInfo bi;
  const int chunk = b % a.nchunk;
  const int row = b / a.nchunk;
  const int cy = row % a.ny, cz = row / a.ny;
  bi.cx0 = chunk * CB;
  bi.m = min(CB, a.nx - bi.cx0);
  bi.Wm = bi.m * K + 1;
  bi.gbase = bi.cx0 * K + a.Mx * (cy * K + a.My * (cz * K));
  bi.xlo = bi.cx0 == 0;
  bi.xhi = bi.cx0 + bi.m == a.nx;
  bi.eflags = (cy == 0 ? 1 : 0) | (cy == a.ny - 1 ? 2 : 0) | (cz == 0 ? 4 : 0) | (cz == a.nz - 1 ? 8 : 0);
  return bi;
}

__device__ __forceinline__ bool tile_boundary(const BatchInfo& bi, int dy, int x) {
  return ((dy >> 23) & bi.eflags) != 0 || (x == 0 && bi.xlo) || (x == bi.Wm - 1 && bi.xhi);
}

template <int N, typename Real, int CB>
__global__ void __launch_bounds__(BrickShape<N, CB>::THREADS,
                                  (sizeof(Real) == 4 ? (1024 / BrickShape<N, CB>::THREADS > 0 ? 1024 / BrickShape<N, CB>::THREADS : 1) : 1))
    brick_vmult_kernel(const __grid_constant__ BrickArgs<N, Real> a, const Real* __restrict__ src,
                       Real* __restrict__ dst) {
  using Sh = BrickShape<N, CB>;
  constexpr int K = Sh::K, NP = Sh::NP, P2 = Sh::P2, CELL = Sh::CELL, N3 = N * N * N;
  constexpr bool PREFETCH = 6 * N * (int)sizeof(Real) / 4 <= 32;
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // Tile descriptors (independent of the batch): element e of the (CB K + 1) x N x N lattice tile
  //   w0 = lattice offset x + Mx (a2 + My a3) relative to the batch's first point,
  //   w1 = cube slot of the element | shared-with-previous-cell bit << 14 | x << 15 | edge flags << 23.
  int2* table = reinterpret_cast<int2*>(smem_raw);
  Real* A = reinterpret_cast<Real*>(smem_raw + Sh::TABLE_BYTES);
  Real* B = A + Sh::CUBES;
  Real* C = B + Sh::CUBES;
  const int t = threadIdx.x;
  for (int e = t; e < Sh::TILE; e += Sh::THREADS) {
    const int rr = e / Sh::WMAX, x = e - rr * Sh::WMAX;
    const int a2 = rr % N, a3 = rr / N;
    const int cc = x / K, a1 = x - cc * K;
    const int off = a3 * P2 + a2 * NP;
    // the last point of a row belongs to the last cell only (slot of cell cc - 1, node K)
    const int slot = cc < CB ? cc * CELL + off + a1 : (cc - 1) * CELL + off + K;
    const int shared_prev = (a1 == 0 && cc >= 1 && cc < CB) ? 1 : 0;
    const int flags = (a2 == 0 ? 1 : 0) | (a2 == K ? 2 : 0) | (a3 == 0 ? 4 : 0) | (a3 == K ? 8 : 0);
    table[e] = make_int2(x + a.Mx * (a2 + a.My * a3), slot | (shared_prev << 14) | (x << 15) | (flags << 23));
  }
  __syncthreads();

  const int c = t % CB;
  const int r = t / CB;
  const int f = r % N, s = r / N;
  const bool line_ok = t < Sh::LINES;
  // line bases
  const int xa2 = Sh::XSWAP ? s : f, xa3 = Sh::XSWAP ? f : s;
  const int xbase = c * CELL + xa3 * P2 + xa2 * NP;  // x-line (a2, a3), stride 1
  const int ybase = c * CELL + s * P2 + f;          // y-line (a1 = f, a3 = s), stride NP
  const int zbase = c * CELL + s * NP + f;          // z-line (a1 = f, a2 = s), stride P2
  const int n_batches = (int)a.n_batches;

  // tile values of the next batch, loaded one batch ahead (Dirichlet points read as 0)
  Real pre[Sh::TILE_ITERS];
  auto load_tile = [&](int bb) {
    const BatchInfo bi = batch_info<CB, K>(a, bb);
#pragma unroll
    for (int it = 0; it < Sh::TILE_ITERS; ++it) {
      const int e = t + it * Sh::THREADS;
      pre[it] = Real(0);
      if (e < Sh::TILE) {
        const int2 d = table[e];
        const int x = (d.y >> 15) & 0xff;
        if (x < bi.Wm && !tile_boundary(bi, d.y, x)) pre[it] = __ldg(src + bi.gbase + d.x);
      }
    }
  };
  if ((int)blockIdx.x < n_batches) load_tile(blockIdx.x);

  for (int b = blockIdx.x; b < n_batches; b += gridDim.x) {
    const BatchInfo bi = batch_info<CB, K>(a, b);
    const int m = bi.m, Wm = bi.Wm;
    const bool act = line_ok && c < m;
    const Real* Gb = a.metric + (int64_t)b * (6 * N3 * CB) + (xa2 * N + xa3 * N * N) * CB + c;

    // 0) the prefetched lattice points of this batch into the cubes
#pragma unroll
    for (int it = 0; it < Sh::TILE_ITERS; ++it) {
      const int e = t + it * Sh::THREADS;
      if (e < Sh::TILE) {
        const int2 d = table[e];
        const int x = (d.y >> 15) & 0xff;
        if (x < Wm) {
          const int slot = d.y & 0x3fff;
          A[slot] = pre[it];
          if ((d.y >> 14) & 1) A[slot - CELL + K] = pre[it];
        }
      }
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
    // next batch's lattice points (consumed after ten phases)
    if (b + (int)gridDim.x < n_batches) load_tile(b + gridDim.x);
    // 1) S along z (in place)
    if (act) {
      Real v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[zbase + j * P2];
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
    // 9) S_z^T
    if (act) {
      Real v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[zbase + j * P2];
      contract_t<N, Real, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[zbase + j * P2] = o[j];
    }
    __syncthreads();
    // 10) scatter: sum shared nodes, coalesced atomic adds; constrained rows copy src
#pragma unroll 4
    for (int e = t; e < Sh::TILE; e += Sh::THREADS) {
      const int2 d = table[e];
      const int x = (d.y >> 15) & 0xff;
      if (x >= Wm) continue;
      const int gi = bi.gbase + d.x;
      const int slot = d.y & 0x3fff;
      if (tile_boundary(bi, d.y, x)) {
        dst[gi] = __ldg(src + gi);
      } else {
        // last point of a partial batch: only the previous (last valid) cell contributes
        Real v = (x == Wm - 1 && m < CB) ? Real(0) : A[slot];
        if ((d.y >> 14) & 1) v += A[slot - CELL + K];
        red_add(dst + gi, v);
      }
    }
    __syncthreads();
  }
}

}  // namespace mfx
