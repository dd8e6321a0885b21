// FP32 brick-row vmult with the tile traffic on the TMA engine.
//
// Same batch decomposition and contraction phases as brick_vmult_kernel
// (vmult_brick.cuh), but the n^2 lattice rows of a batch are moved by the
// Tensor Memory Accelerator: one 1D tensor copy per row into shared memory
// (tracked by an mbarrier, issued one batch ahead into a second buffer) and
// one 1D tensor reduce-add per row from shared memory into dst.  Rows start
// at arbitrary DoF offsets, so each copy starts at the 16-byte boundary
// below the row and the row sits at offset (start mod 4) inside its tile
// row.  Dirichlet points are masked in registers by the thread that owns
// the line (values read as 0; results written as 0, so the reduce adds 0 and
// the constrained rows keep dst = src from the boundary-copy kernel).
// Points of a tile row outside the batch are kept at 0 in the output tile.
// Every wait on an mbarrier is bounded (about one second of clock); a
// timeout sets an error word, drains the CTA's outstanding copies and ends
// the CTA.
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
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

template <int N, int CB>
__global__ void __launch_bounds__(BrickShape<N, CB, float>::THREADS,
                                  (1024 / BrickShape<N, CB, float>::THREADS > 0 ? 1024 / BrickShape<N, CB, float>::THREADS : 1))
    brick_vmult_tma_kernel(const __grid_constant__ TmaArgs<N> a) {
  using Sh = BrickShape<N, CB, float>;
  using Tm = TmaShape<N, CB>;
  constexpr int K = Sh::K, NP = Sh::NP, P2 = Sh::P2, CELL = Sh::CELL, N3 = N * N * N;
  constexpr int PITCH = Tm::PITCH, ROWS = Tm::ROWS, BOX = Tm::BOX;
  constexpr bool PREFETCH = 6 * N <= 32;
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* in_tiles = reinterpret_cast<float*>(smem_raw);  // 2 x TILE
  float* out_tiles = in_tiles + 2 * Tm::TILE;            // 2 x TILE
  float* A = out_tiles + 2 * Tm::TILE;
  float* B = A + Sh::CUBES;
  float* C = B + Sh::CUBES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(C + Sh::CUBES + ((Sh::CUBES & 1) ? 1 : 0));

  const int t = threadIdx.x;
  const int c = t % CB;
  const int r = t / CB;
  const int f = r % N, s = r / N;
  const bool line_ok = t < Sh::LINES;
  const int xa2 = Sh::XSWAP ? s : f, xa3 = Sh::XSWAP ? f : s;
  const int xbase = c * CELL + xa3 * P2 + xa2 * NP;
  const int ybase = c * CELL + s * P2 + f;
  const int zbase = c * CELL + s * NP + f;
  const int zx = c * K + f;  // tile point of this thread's z-line
  // the TMA work (row copies, reduces, padding) goes to the last warp, which has idle lanes
  const int lane = t & 31;
  const bool tma_warp = (t >> 5) == Sh::THREADS / 32 - 1;

  if (t == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  for (int i = t; i < 2 * Tm::TILE; i += Sh::THREADS) out_tiles[i] = 0.0f;
  fence_proxy_async();
  __syncthreads();

  // TMA warp: copies of batch bb into input tile buffer `buf`, lane l issues rows l, l + 32, ...
  auto issue_loads = [&](int bb, int buf) {
    const BatchInfo bi = batch_info<CB, K>(a, bb);
    fence_proxy_async();
    if (lane == 0) mbar_arrive_expect_tx(&bars[buf], ROWS * BOX * 4);
    __syncwarp();
    float* T = in_tiles + buf * Tm::TILE;
    for (int row = lane; row < ROWS; row += 32) {
      const int a2 = row % N, a3 = row / N;
      const int gi0 = bi.gbase + a.Mx * (a2 + a.My * a3);
      tma_load_1d(T + row * PITCH, &a.tsrc, gi0 & ~3, &bars[buf]);
    }
  };

  int it = 0;
  bool failed = false, next_issued = false;
  if (tma_warp && (int)blockIdx.x < a.n_batches) issue_loads(blockIdx.x, 0);

  for (int b = blockIdx.x; b < a.n_batches; b += gridDim.x, ++it) {
    const int buf = it & 1;
    const BatchInfo bi = batch_info<CB, K>(a, b);
    const int m = bi.m;
    const bool act = line_ok && c < m;
    const float* Gb = a.metric + (int64_t)b * (6 * N3 * CB) + (xa2 * N + xa3 * N * N) * CB + c;
    float* T = in_tiles + buf * Tm::TILE;
    float* O = out_tiles + buf * Tm::TILE;
    // row start offsets (mod 4) of this thread's z-line rows: rows a3 N + s, a3 = 0..K
    const int zrow0 = bi.gbase + a.Mx * s;  // + Mx My a3
    // Dirichlet mask of this z-line: whole line, or its first / last point
    const bool lbnd = (zx == 0 && bi.xlo) || (zx == bi.Wm - 1 && bi.xhi) || (s == 0 && (bi.eflags & 1)) ||
                      (s == K && (bi.eflags & 2));
    const bool zlo = (bi.eflags & 4) != 0, zhi = (bi.eflags & 8) != 0;

    next_issued = b + (int)gridDim.x < a.n_batches;
    if (tma_warp && next_issued) issue_loads(b + gridDim.x, buf ^ 1);
    float G[PREFETCH ? 6 : 1][N];
    if (PREFETCH && act) {
#pragma unroll
      for (int e = 0; e < 6; ++e)
#pragma unroll
        for (int q = 0; q < N; ++q) G[e][q] = __ldg(Gb + (e * N3 + q) * CB);
    }
    const bool ok = mbar_wait(&bars[buf], (it >> 1) & 1);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    // 1) S along z: z-lines from the tile (Dirichlet points read as 0)
    if (act) {
      float v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const int g = zrow0 + a.Mx * a.My * j;
        v[j] = T[(j * N + s) * PITCH + (g & 3) + zx];
      }
      if (lbnd) {
#pragma unroll
        for (int j = 0; j < N; ++j) v[j] = 0.0f;
      }
      if (zlo) v[0] = 0.0f;
      if (zhi) v[K] = 0.0f;
      contract<N, float, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[zbase + j * P2] = o[j];
    }
    __syncthreads();
    // 2) S along y
    if (act) {
      float v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[ybase + j * NP];
      contract<N, float, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[ybase + j * NP] = o[j];
    }
    __syncthreads();
    // 3) S along x -> values at Gauss points; D along x in registers
    float g1[N];
    if (act) {
      float v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[xbase + j];
      contract<N, float, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[xbase + j] = o[j];
      contract<N, float, MAT_D>(o, g1);
    }
    __syncthreads();
    // 4) D along y -> B, D along z -> C
    if (act) {
      float v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[ybase + j * NP];
      contract<N, float, MAT_D>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) B[ybase + j * NP] = o[j];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[zbase + j * P2];
      contract<N, float, MAT_D>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) C[zbase + j * P2] = o[j];
    }
    __syncthreads();
    // 5) quadrature-point metric on the x-line; D_x^T in registers
    float t1[N];
    if (act) {
      float h1[N];
#pragma unroll
      for (int q = 0; q < N; ++q) {
        float G00, G01, G02, G11, G12, G22;
        if constexpr (PREFETCH) {
          G00 = G[0][q]; G01 = G[1][q]; G02 = G[2][q]; G11 = G[3][q]; G12 = G[4][q]; G22 = G[5][q];
        } else {
          G00 = __ldg(Gb + (0 * N3 + q) * CB); G01 = __ldg(Gb + (1 * N3 + q) * CB);
          G02 = __ldg(Gb + (2 * N3 + q) * CB); G11 = __ldg(Gb + (3 * N3 + q) * CB);
          G12 = __ldg(Gb + (4 * N3 + q) * CB); G22 = __ldg(Gb + (5 * N3 + q) * CB);
        }
        const float u1 = g1[q], u2 = B[xbase + q], u3 = C[xbase + q];
        h1[q] = G00 * u1 + G01 * u2 + G02 * u3;
        B[xbase + q] = G01 * u1 + G11 * u2 + G12 * u3;
        C[xbase + q] = G02 * u1 + G12 * u2 + G22 * u3;
      }
      contract_t<N, float, MAT_D>(h1, t1);
    }
    __syncthreads();
    // 6) D_y^T on B, D_z^T on C
    if (act) {
      float v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = B[ybase + j * NP];
      contract_t<N, float, MAT_D>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) B[ybase + j * NP] = o[j];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = C[zbase + j * P2];
      contract_t<N, float, MAT_D>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) C[zbase + j * P2] = o[j];
    }
    __syncthreads();
    // 7) sum of the three components, S_x^T -> A
    if (act) {
      float v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = t1[j] + B[xbase + j] + C[xbase + j];
      contract_t<N, float, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[xbase + j] = o[j];
    }
    __syncthreads();
    // 8) S_y^T; the output buffer of this batch was last read by the reduces issued two
    //    batches ago: make sure they are done before step 9 rewrites it
    if (tma_warp) bulk_wait_read<1>();
    if (act) {
      float v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[ybase + j * NP];
      contract_t<N, float, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[ybase + j * NP] = o[j];
    }
    __syncthreads();
    // 9) S_z^T into the output tile: a1 < K nodes first, then the a1 = K nodes add to the
    //    next cell's a1 = 0 node (the last valid cell stores); warp 0 clears the points of each
    //    tile row outside the batch
    float o9[N];
    if (act) {
      float v[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[zbase + j * P2];
      contract_t<N, float, MAT_S>(v, o9);
      if (lbnd) {
#pragma unroll
        for (int j = 0; j < N; ++j) o9[j] = 0.0f;
      }
      if (zlo) o9[0] = 0.0f;
      if (zhi) o9[K] = 0.0f;
      if (f < K) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const int g = zrow0 + a.Mx * a.My * j;
          O[(j * N + s) * PITCH + (g & 3) + zx] = o9[j];
        }
      }
    }
    if (tma_warp) {
      for (int row = lane; row < ROWS; row += 32) {
        const int a2 = row % N, a3 = row / N;
        const int off = (bi.gbase + a.Mx * (a2 + a.My * a3)) & 3;
        float* p = O + row * PITCH;
        for (int x = 0; x < off; ++x) p[x] = 0.0f;
        for (int x = off + bi.Wm; x < BOX; ++x) p[x] = 0.0f;
      }
    }
    __syncthreads();
    if (act && f == K) {
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const int g = zrow0 + a.Mx * a.My * j;
        float* p = O + (j * N + s) * PITCH + (g & 3) + zx;
        if (c < m - 1)
          *p += o9[j];
        else
          *p = o9[j];
      }
    }
    fence_proxy_async();
    __syncthreads();
    // 10) TMA warp: reduce-add the output rows into dst (one bulk group per lane and batch)
    if (tma_warp) {
      for (int row = lane; row < ROWS; row += 32) {
        const int a2 = row % N, a3 = row / N;
        const int gi0 = bi.gbase + a.Mx * (a2 + a.My * a3);
        tma_reduce_add_1d(&a.tdst, gi0 & ~3, O + row * PITCH);
      }
      bulk_commit();
    }
  }
  if (tma_warp) bulk_wait_all();
  if (failed) {
    if (tma_warp && lane == 0) {
      atomicExch(a.err, 1);
      // drain the copies that may still be in flight before the CTA ends (bounded)
      const int buf = it & 1;
      mbar_wait(&bars[buf], (unsigned)((it >> 1) & 1));
      if (next_issued) mbar_wait(&bars[buf ^ 1], (unsigned)(((it + 1) >> 1) & 1));
    }
  }
}

}  // namespace mfx
