// FP32 brick-row vmult on pairs of cells with packed FP32 arithmetic.
//
// Per batch of CB cells of one row: the batch's n^2 lattice rows are copied into a shared-memory tile
// by TMA one batch ahead (vmult_brick_tma.cuh); forward contractions S_z (z-lines read straight from
// the tile, Dirichlet points as 0), S_y, S_x, then D_x (registers), D_y, D_z; h = G_q grad at every
// Gauss point with G prefetched into registers; transposed contractions summed over the components,
// S_x^T, S_y^T, and S_z^T into an output tile (nodes shared by neighbouring cells in two passes),
// which is added to dst by TMA reduce-adds (dst holds src on Dirichlet rows and 0 elsewhere before
// the launch).  Every thread owns the
// same line of two neighbouring cells (2c, 2c + 1) of the batch, held as a float pair: each
// contraction is a chain of packed FMAs (two FMAs per instruction, Blackwell FFMA2), shared-memory
// accesses move 8 bytes, and the per-line index and control work is shared by two cells.  The
// cube paddings of CB / 2 float pairs are those of CB single cells (the bank-conflict search
// gives the same optimum for 8-byte elements in half-warp phases).
#pragma once

#include "vmult_brick_tma.cuh"

namespace mfx {

template <int N, int CB>
struct PairShape {
  static constexpr int LINES = (CB / 2) * N * N;
  static constexpr int THREADS = (LINES + 31) / 32 * 32;
  static constexpr int CUBES = (CB / 2) * BrickShape<N, CB, float>::CELL;  // float2 elements per cube
  // resident CTAs per SM the register budget is sized for (fewer for the larger degrees)
  static constexpr int MIN_BLOCKS = (N == 2 || N == 4) ? (512 / THREADS > 0 ? 512 / THREADS : 1)
                                                      : (768 / THREADS > 0 ? 768 / THREADS : 1);
  static constexpr size_t SMEM =
      (size_t)4 * TmaShape<N, CB>::TILE * sizeof(float) + 3 * (size_t)CUBES * sizeof(float2) + 2 * sizeof(uint64_t);
};

template <int N, int MAT>
__device__ __forceinline__ void contract2(const float2 (&in)[N], float2 (&out)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const float m0 = (float)basis_entry<N, MAT>(i * N);
    float2 s = __fmul2_rn(make_float2(m0, m0), in[0]);
#pragma unroll
    for (int j = 1; j < N; ++j) {
      const float mj = (float)basis_entry<N, MAT>(i * N + j);
      s = __ffma2_rn(make_float2(mj, mj), in[j], s);
    }
    out[i] = s;
  }
}

template <int N, int MAT>
__device__ __forceinline__ void contract2_t(const float2 (&in)[N], float2 (&out)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const float m0 = (float)basis_entry<N, MAT>(i);
    float2 s = __fmul2_rn(make_float2(m0, m0), in[0]);
#pragma unroll
    for (int j = 1; j < N; ++j) {
      const float mj = (float)basis_entry<N, MAT>(j * N + i);
      s = __ffma2_rn(make_float2(mj, mj), in[j], s);
    }
    out[i] = s;
  }
}

template <int N, int CB, bool BOXM = false>
__global__ void __launch_bounds__(PairShape<N, CB>::THREADS, PairShape<N, CB>::MIN_BLOCKS)
    brick_vmult_tma2_kernel(const __grid_constant__ TmaArgs<N> a) {
  using Sh = BrickShape<N, CB, float>;  // cube paddings of CB cells = paddings of CB / 2 float pairs
  using Tm = TmaShape<N, CB>;
  using Ps = PairShape<N, CB>;
  constexpr int PP = CB / 2;
  constexpr int K = Sh::K, NP = Sh::NP, P2 = Sh::P2, CELL = Sh::CELL, N3 = N * N * N;
  constexpr int PITCH = Tm::PITCH, ROWS = Tm::ROWS, BOX = Tm::BOX;
  // k = 1, 3: the metric of a thread's x-line in registers (6 N float pairs), loaded ahead of its use.
  // k = 2, 4: loaded where it is used, from L2 (the TMA engine prefetches each batch's metric one batch
  // ahead, below), which frees registers for more CTAs per SM: Q4 on 64^3 0.2871 -> 0.2708 ms, Q2 on
  // 128^3 0.3903 -> 0.3814 ms (Q3 measured slower that way: 0.304 -> 0.314 ms)
  constexpr bool PREFETCH = !BOXM && (N == 2 || N == 4);
  // k = 1: the next batch's metric is requested right after the current one is used (spreads the
  // metric stream over the whole batch); k = 3: at the start of the batch
  constexpr bool XPREF = PREFETCH && N <= 3;
  // L2 prefetch of the metric one batch ahead for k >= 2 (k = 8: 0.949 -> 0.863 ms on 40^3, Q3 on 86^3
  // 0.310 -> 0.304); with the register prefetch of k = 1 it measured slower
  constexpr int MDIST = (!BOXM && N >= 3) ? 1 : 0;  // box cells read three entries of each line
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* in_tiles = reinterpret_cast<float*>(smem_raw);  // 2 x TILE
  float* out_tiles = in_tiles + 2 * Tm::TILE;            // 2 x TILE
  float2* A = reinterpret_cast<float2*>(out_tiles + 2 * Tm::TILE);
  float2* B = A + Ps::CUBES;
  float2* C = B + Ps::CUBES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(C + Ps::CUBES);

  const int t = threadIdx.x;
  const int c = t % PP;  // pair: cells 2c and 2c + 1 of the batch
  const int r = t / PP;
  const int f = r % N, s = r / N;
  const bool line_ok = t < Ps::LINES;
  const int xa2 = Sh::XSWAP ? s : f, xa3 = Sh::XSWAP ? f : s;
  const int xbase = c * CELL + xa3 * P2 + xa2 * NP;
  const int ybase = c * CELL + s * P2 + f;
  const int zbase = c * CELL + s * NP + f;
  const int zx = 2 * c * K + f;  // tile point of this thread's z-line in the first cell of the pair; + K for the second
  // the TMA work (row copies, reduces, padding) goes to the last warp, which has idle lanes
  const int lane = t & 31;
  const bool tma_warp = (t >> 5) == Ps::THREADS / 32 - 1;

  if (t == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  for (int i = t; i < 2 * Tm::TILE; i += Ps::THREADS) out_tiles[i] = 0.0f;
  fence_proxy_async();
  __syncthreads();

  // TMA warp: copies of the batch at position pb into input tile buffer `buf`, lane l issues rows
  // l, l + 32, ...
  auto issue_loads = [&](const BatchPos& pb, int buf) {
    const BatchInfo bi = batch_info_at<CB, K>(a, pb);
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
  BatchPos pos = batch_pos(a, blockIdx.x);
  if (tma_warp && (int)blockIdx.x < a.n_batches) issue_loads(pos, 0);
  // metric of the batch in registers (XPREF: requested during the previous batch, right after that
  // batch's own metric was used); entries of pairs outside a partial batch lie inside the padded
  // layout and are unused
  const float2* Gthread = reinterpret_cast<const float2*>(a.metric + (xa2 * N + xa3 * N * N) * CB + 2 * c);
  float2 G[PREFETCH ? 6 : 1][N];
  if (XPREF && line_ok && (int)blockIdx.x < a.n_batches) {
    const float2* G0 = Gthread + (int64_t)blockIdx.x * (6 * N3 * CB) / 2;
#pragma unroll
    for (int e = 0; e < 6; ++e)
#pragma unroll
      for (int q = 0; q < N; ++q) G[e][q] = __ldg(G0 + (e * N3 + q) * PP);
  }

  for (int b = blockIdx.x; b < a.n_batches; b += gridDim.x, ++it) {
    const int buf = it & 1;
    const BatchInfo bi = batch_info_at<CB, K>(a, pos);
    const int m = bi.m;
    const bool act = line_ok && 2 * c < m;       // first cell of the pair valid
    const bool act1 = line_ok && 2 * c + 1 < m;  // second cell valid
    const float2* Gb =
        reinterpret_cast<const float2*>(a.metric + (int64_t)b * (6 * N3 * CB) + (xa2 * N + xa3 * N * N) * CB + 2 * c);
    float* T = in_tiles + buf * Tm::TILE;
    float* O = out_tiles + buf * Tm::TILE;
    // row start offsets (mod 4) of this thread's z-line rows: rows a3 N + s, a3 = 0..K
    const int zrow0 = bi.gbase + a.Mx * s;  // + Mx My a3
    // Dirichlet mask of this z-line: whole line, or its first / last point
    const bool ebnd = (s == 0 && (bi.eflags & 1)) || (s == K && (bi.eflags & 2));
    const bool lbnd0 = ebnd || (zx == 0 && bi.xlo) || (zx == bi.Wm - 1 && bi.xhi);
    const bool lbnd1 = ebnd || (zx + K == 0 && bi.xlo) || (zx + K == bi.Wm - 1 && bi.xhi);
    const bool zlo = (bi.eflags & 4) != 0, zhi = (bi.eflags & 8) != 0;

    next_issued = b + (int)gridDim.x < a.n_batches;
    if (tma_warp && next_issued) {
      BatchPos next = pos;
      batch_advance(next, a);
      issue_loads(next, buf ^ 1);
    }
    // the metric of this CTA's batch MDIST batches ahead is brought into L2 by the TMA engine, so the
    // register loads of that batch hit L2 and the HBM stream of the metric, which is most of the bytes,
    // overlaps the batches in between without holding registers
    if (MDIST > 0 && tma_warp && lane < 3) {
      const int bn = b + MDIST * (int)gridDim.x;
      if (bn < a.n_batches) {
        constexpr unsigned BYTES = 6u * N3 * CB * 4u;  // one batch of the metric, contiguous
        constexpr unsigned CHUNK = (BYTES / 3 + 15u) & ~15u;
        const unsigned off = lane * CHUNK;
        if (off < BYTES)
          prefetch_l2_bulk(reinterpret_cast<const char*>(a.metric + (int64_t)bn * (6 * N3 * CB)) + off,
                           off + CHUNK <= BYTES ? CHUNK : BYTES - off);
      }
    }
    if (PREFETCH && !XPREF && act) {
      const float2* G0 = Gthread + (int64_t)b * (6 * N3 * CB) / 2;
#pragma unroll
      for (int e = 0; e < 6; ++e)
#pragma unroll
        for (int q = 0; q < N; ++q) G[e][q] = __ldg(G0 + (e * N3 + q) * PP);
    }
    const bool ok = mbar_wait(&bars[buf], (it >> 1) & 1);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    // 1) S along z: z-lines from the tile (Dirichlet points read as 0)
    if (act) {
      float2 v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const int g = zrow0 + a.Mx * a.My * j;
        const float* row = T + (j * N + s) * PITCH + (g & 3) + zx;
        v[j] = make_float2(lbnd0 ? 0.0f : row[0], lbnd1 ? 0.0f : row[K]);
      }
      if (zlo) v[0] = make_float2(0.0f, 0.0f);
      if (zhi) v[K] = make_float2(0.0f, 0.0f);
      contract2<N, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[zbase + j * P2] = o[j];
    }
    __syncthreads();
    // 2) S along y
    if (act) {
      float2 v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[ybase + j * NP];
      contract2<N, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[ybase + j * NP] = o[j];
    }
    __syncthreads();
    // 3) S along x -> values at Gauss points; D along x in registers
    float2 g1[N];
    if (act) {
      float2 v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[xbase + j];
      contract2<N, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[xbase + j] = o[j];
      contract2<N, MAT_D>(o, g1);
    }
    __syncthreads();
    // 4) D along y -> B, D along z -> C
    if (act) {
      float2 v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[ybase + j * NP];
      contract2<N, MAT_D>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) B[ybase + j * NP] = o[j];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[zbase + j * P2];
      contract2<N, MAT_D>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) C[zbase + j * P2] = o[j];
    }
    __syncthreads();
    // 5) quadrature-point metric on the x-line; D_x^T in registers
    float2 t1[N];
    if (act) {
      float2 h1[N];
      if constexpr (BOXM) {
        // box cells: the metric on the line is w_q / w_0 times its first point's diagonal
        const float2 D0 = __ldg(Gb), D1 = __ldg(Gb + 3 * N3 * PP), D2 = __ldg(Gb + 5 * N3 * PP);
#pragma unroll
        for (int q = 0; q < N; ++q) {
          const float2 rq = make_float2(a.wr[q], a.wr[q]);
          const float2 u1 = g1[q], u2 = B[xbase + q], u3 = C[xbase + q];
          h1[q] = __fmul2_rn(__fmul2_rn(rq, D0), u1);
          B[xbase + q] = __fmul2_rn(__fmul2_rn(rq, D1), u2);
          C[xbase + q] = __fmul2_rn(__fmul2_rn(rq, D2), u3);
        }
      } else {
#pragma unroll
      for (int q = 0; q < N; ++q) {
        float2 G00, G01, G02, G11, G12, G22;
        if constexpr (PREFETCH) {
          G00 = G[0][q]; G01 = G[1][q]; G02 = G[2][q]; G11 = G[3][q]; G12 = G[4][q]; G22 = G[5][q];
        } else {
          G00 = __ldg(Gb + (0 * N3 + q) * PP); G01 = __ldg(Gb + (1 * N3 + q) * PP);
          G02 = __ldg(Gb + (2 * N3 + q) * PP); G11 = __ldg(Gb + (3 * N3 + q) * PP);
          G12 = __ldg(Gb + (4 * N3 + q) * PP); G22 = __ldg(Gb + (5 * N3 + q) * PP);
        }
        const float2 u1 = g1[q], u2 = B[xbase + q], u3 = C[xbase + q];
        h1[q] = __ffma2_rn(G02, u3, __ffma2_rn(G01, u2, __fmul2_rn(G00, u1)));
        B[xbase + q] = __ffma2_rn(G12, u3, __ffma2_rn(G11, u2, __fmul2_rn(G01, u1)));
        C[xbase + q] = __ffma2_rn(G22, u3, __ffma2_rn(G12, u2, __fmul2_rn(G02, u1)));
      }
      }
      contract2_t<N, MAT_D>(h1, t1);
    }
    if (XPREF && line_ok && b + (int)gridDim.x < a.n_batches) {  // the next batch's metric
      const float2* Gn = Gthread + (int64_t)(b + gridDim.x) * (6 * N3 * CB) / 2;
#pragma unroll
      for (int e = 0; e < 6; ++e)
#pragma unroll
        for (int q = 0; q < N; ++q) G[e][q] = __ldg(Gn + (e * N3 + q) * PP);
    }
    __syncthreads();
    // 6) D_y^T on B, D_z^T on C
    if (act) {
      float2 v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = B[ybase + j * NP];
      contract2_t<N, MAT_D>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) B[ybase + j * NP] = o[j];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = C[zbase + j * P2];
      contract2_t<N, MAT_D>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) C[zbase + j * P2] = o[j];
    }
    __syncthreads();
    // 7) sum of the three components, S_x^T -> A
    if (act) {
      float2 v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = __fadd2_rn(__fadd2_rn(t1[j], B[xbase + j]), C[xbase + j]);
      contract2_t<N, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[xbase + j] = o[j];
    }
    __syncthreads();
    // 8) S_y^T; the output buffer of this batch was last read by the reduces issued two
    //    batches ago: make sure they are done before step 9 rewrites it
    if (tma_warp) bulk_wait_read<1>();
    if (act) {
      float2 v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[ybase + j * NP];
      contract2_t<N, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[ybase + j * NP] = o[j];
    }
    __syncthreads();
    // 9) S_z^T into the output tile: a1 < K nodes first, then the a1 = K nodes add to the
    //    next cell's a1 = 0 node (the last valid cell stores); warp 0 clears the points of each
    //    tile row outside the batch
    float2 o9[N];
    if (act) {
      float2 v[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[zbase + j * P2];
      contract2_t<N, MAT_S>(v, o9);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        if (lbnd0) o9[j].x = 0.0f;
        if (lbnd1 || !act1) o9[j].y = 0.0f;
      }
      if (zlo) o9[0] = make_float2(0.0f, 0.0f);
      if (zhi) o9[K] = make_float2(0.0f, 0.0f);
      if (f < K) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const int g = zrow0 + a.Mx * a.My * j;
          float* row = O + (j * N + s) * PITCH + (g & 3) + zx;
          row[0] = o9[j].x;
          if (act1) row[K] = o9[j].y;
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
    // a1 = K nodes: the first cell's goes to the second cell's a1 = 0 node (stored if the second
    // cell is not in the batch), the second cell's to the next pair's first cell (or stored)
    if (act && f == K) {
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const int g = zrow0 + a.Mx * a.My * j;
        float* row = O + (j * N + s) * PITCH + (g & 3) + zx;
        if (act1)
          row[0] += o9[j].x;
        else
          row[0] = o9[j].x;
        if (act1) {
          if (2 * c + 2 < m)
            row[K] += o9[j].y;
          else
            row[K] = o9[j].y;
        }
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
    batch_advance(pos, a);
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
