// FP32 vmult on meshes with index tables (octrees, hanging nodes), pairs of cells per thread: the
// operator of Sec. 3.6 on locally refined meshes, with the hanging-node constraints of Sec. 3.1 and
// Fig. 2 resolved in the gather and its transpose in the scatter (Sec. 3.3).
//
// The compute structure is that of brick_vmult_tma2_kernel: a CTA takes batches of CB consecutive
// cells (the Morton order keeps them close in space), every thread owns the same 1D line of two
// neighbouring cells (2c, 2c + 1) as a float pair, contractions are packed FFMA2 chains on
// conflict-free padded cubes, and the metric (interleaved per batch, [batch][6][q][CB]) is
// prefetched into registers a phase group ahead.  What differs is the gather and the scatter: the
// batch's cell index table (CB n^3 int32, contiguous) is staged in shared memory once per batch, the
// z-line values are read from src through it with the constraints resolved per node (a hanging
// node is the weighted sum of its masters, a Dirichlet node reads as 0), and the results are added
// into dst with atomics through the same table (hanging nodes into their masters with the same
// weights, Dirichlet nodes dropped).  dst must hold src on constrained rows and 0 elsewhere before
// the launch (vmult_prologue).
#pragma once

#include "vmult.cuh"
#include "vmult_brick_tma2.cuh"

namespace mfx {

// Degrees (N = k + 1) whose FP32 octree vmult uses this kernel, by measurement on 4-5M DoF octrees with
// hanging nodes (ms, this kernel / per-cell kernel): k = 1 0.059 / 0.061, k = 8 1.05 / 1.45; for
// k = 2..7 the per-cell kernel (vmult_kernel), whose cell-major lanes coalesce the gather and the
// scatter, is faster (k = 4: 0.317 / 0.242).
template <int N>
struct OctreePairFor {
  static constexpr bool value = N == 2 || N == 9;
};

template <int N>
struct OctreePairArgs {
  const float* metric;       // FP32 metric, [batch][6][N^3][CB]
  const int32_t* cell_dofs;  // n_cells x N^3, >= 0 free DoF, < 0: -(row + 1) into the constraint rows
  const int64_t* cptr;
  const int32_t* cmaster;
  const float* cweight;
  int64_t n_cells;
  int n_batches;
  const int32_t* skip;
  // box cells: metric w_q diag(box[cell][0..2]), wq the 1D Gauss weights (BOX variant)
  const float* box;
  float wq[N];
};

template <int N, int CB>
struct OctreePairShape {
  static constexpr int N3 = N * N * N;
  static constexpr int IDX = CB * N3;  // staged index table entries
  static constexpr size_t SMEM = 3 * (size_t)PairShape<N, CB>::CUBES * sizeof(float2) + (size_t)IDX * sizeof(int32_t);
};

// Value of one local node: free DoF, weighted masters (hanging) or 0 (Dirichlet).
__device__ __forceinline__ float gather_node(const int32_t e, const float* __restrict__ src, const int64_t* cptr,
                                             const int32_t* cmaster, const float* cweight) {
  if (e >= 0) return __ldg(src + e);
  const int32_t row = -e - 1;
  float s = 0.0f;
  for (int64_t p = __ldg(cptr + row), pe = __ldg(cptr + row + 1); p < pe; ++p)
    s = __fmaf_rn(__ldg(cweight + p), __ldg(src + __ldg(cmaster + p)), s);
  return s;
}

// Transpose of gather_node.
__device__ __forceinline__ void scatter_node(const int32_t e, float v, float* __restrict__ dst, const int64_t* cptr,
                                             const int32_t* cmaster, const float* cweight) {
  if (e >= 0) {
    atomicAdd(dst + e, v);
    return;
  }
  const int32_t row = -e - 1;
  for (int64_t p = __ldg(cptr + row), pe = __ldg(cptr + row + 1); p < pe; ++p)
    atomicAdd(dst + __ldg(cmaster + p), __ldg(cweight + p) * v);
}

template <int N, int CB, bool BOX = false>
__global__ void __launch_bounds__(PairShape<N, CB>::THREADS, PairShape<N, CB>::MIN_BLOCKS)
    octree_vmult_pair_kernel(const __grid_constant__ OctreePairArgs<N> a, const float* __restrict__ src,
                             float* __restrict__ dst) {
  using Sh = BrickShape<N, CB, float>;  // cube paddings of CB cells = paddings of CB / 2 float pairs
  using Ps = PairShape<N, CB>;
  using Os = OctreePairShape<N, CB>;
  constexpr int PP = CB / 2;
  constexpr int K = Sh::K, NP = Sh::NP, P2 = Sh::P2, CELL = Sh::CELL, N3 = N * N * N;
  constexpr bool PREFETCH = N <= 5 && !BOX;
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* A = reinterpret_cast<float2*>(smem_raw);
  float2* B = A + Ps::CUBES;
  float2* C = B + Ps::CUBES;
  int32_t* idx = reinterpret_cast<int32_t*>(C + Ps::CUBES);

  const int t = threadIdx.x;
  const int c = t % PP;  // pair: cells 2c and 2c + 1 of the batch
  const int r = t / PP;
  const int f = r % N, s = r / N;
  const bool line_ok = t < Ps::LINES;
  const int xa2 = Sh::XSWAP ? s : f, xa3 = Sh::XSWAP ? f : s;
  const int xbase = c * CELL + xa3 * P2 + xa2 * NP;
  const int ybase = c * CELL + s * P2 + f;
  const int zbase = c * CELL + s * NP + f;
  // this thread's z-line (i1 = f, i2 = s) in the staged table: node j at zidx + j N^2 (+ N^3 for 2c + 1)
  const int zidx = 2 * c * N3 + s * N + f;

  for (int b = blockIdx.x; b < a.n_batches; b += gridDim.x) {
    const int64_t cell0 = (int64_t)b * CB;
    const int64_t rest = a.n_cells - cell0;
    const int m = rest < CB ? (int)rest : CB;
    const bool act = line_ok && 2 * c < m;
    const bool act1 = line_ok && 2 * c + 1 < m;
    const float2* Gb = BOX ? nullptr
                           : reinterpret_cast<const float2*>(a.metric + (int64_t)b * (6 * N3 * CB) +
                                                             (xa2 * N + xa3 * N * N) * CB + 2 * c);
    float2 G[PREFETCH ? 6 : 1][N];
    if (PREFETCH && act) {
#pragma unroll
      for (int e = 0; e < 6; ++e)
#pragma unroll
        for (int q = 0; q < N; ++q) G[e][q] = __ldg(Gb + (e * N3 + q) * PP);
    }
    // stage the batch's index table (contiguous, coalesced; the tail of a short batch is not read)
    {
      const int32_t* g = a.cell_dofs + cell0 * N3;
      const int n = m * N3;
      for (int i = t; i < n; i += Ps::THREADS) idx[i] = __ldg(g + i);
    }
    __syncthreads();
    // 1) gather z-lines through the table, S along z
    if (act) {
      float2 v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const float v0 = gather_node(idx[zidx + j * N * N], src, a.cptr, a.cmaster, a.cweight);
        const float v1 = act1 ? gather_node(idx[zidx + N3 + j * N * N], src, a.cptr, a.cmaster, a.cweight) : 0.0f;
        v[j] = make_float2(v0, v1);
      }
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
      if constexpr (BOX) {
        // box cells: metric w_q diag(D) per cell, the pair's two diagonals as the lanes (a missing second
        // cell of a short batch repeats the first)
        const int64_t c0 = cell0 + 2 * c, c1 = act1 ? c0 + 1 : c0;
        const float wyz = a.wq[xa2] * a.wq[xa3];
        const float2 D0 = make_float2(wyz * __ldg(a.box + c0 * 3), wyz * __ldg(a.box + c1 * 3));
        const float2 D1 = make_float2(wyz * __ldg(a.box + c0 * 3 + 1), wyz * __ldg(a.box + c1 * 3 + 1));
        const float2 D2 = make_float2(wyz * __ldg(a.box + c0 * 3 + 2), wyz * __ldg(a.box + c1 * 3 + 2));
#pragma unroll
        for (int q = 0; q < N; ++q) {
          const float2 wx = make_float2(a.wq[q], a.wq[q]);
          const float2 u1 = g1[q], u2 = B[xbase + q], u3 = C[xbase + q];
          h1[q] = __fmul2_rn(__fmul2_rn(wx, D0), u1);
          B[xbase + q] = __fmul2_rn(__fmul2_rn(wx, D1), u2);
          C[xbase + q] = __fmul2_rn(__fmul2_rn(wx, D2), u3);
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
    // 8) S_y^T
    if (act) {
      float2 v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[ybase + j * NP];
      contract2_t<N, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[ybase + j * NP] = o[j];
    }
    __syncthreads();
    // 9) S_z^T and scatter through the table
    if (act) {
      float2 v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[zbase + j * P2];
      contract2_t<N, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        scatter_node(idx[zidx + j * N * N], o[j].x, dst, a.cptr, a.cmaster, a.cweight);
        if (act1) scatter_node(idx[zidx + N3 + j * N * N], o[j].y, dst, a.cptr, a.cmaster, a.cweight);
      }
    }
    __syncthreads();  // the table and the cubes are rewritten by the next batch
  }
}

}  // namespace mfx
