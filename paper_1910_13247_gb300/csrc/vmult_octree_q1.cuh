// FP32 octree vmult at k = 1 on box cells (the metric one diagonal per cell): the operator of Sec. 3.6
// with the tensor-product evaluation of Sec. 3.1 (two Gauss points per direction) in registers, one
// thread per cell, and the constraints of Sec. 3.3 resolved in the gather and its transpose in the
// scatter.
//
// At k = 1 a cell has eight nodes and every node is shared, so the vmult is bound by the random gathers
// and scatter atomics of the index table (about eight of each per DoF), not by arithmetic.  The eight
// children of an octant are consecutive leaves (leaves are sorted by Morton code) and touch only 27
// distinct nodes: the setup finds the octants in the cell order and stores their 27 node entries; the
// kernel gathers each of the 27 once into shared memory, the octant's eight threads add their results
// there, and 27 scatters (not 64) go to dst.  The cells outside octants gather and scatter per node.
// dst must hold src on the constrained rows and 0 elsewhere before the launch (vmult_prologue).
#pragma once

#include <climits>

#include "vmult_octree2.cuh"

namespace mfx {

// Octants: cells i .. i + 7 with child c at (c & 1, (c >> 1) & 1, c >> 2) of the 2 x 2 x 2 block (the
// Morton order, x fastest) and its local node (i1, i2, i3) (index i1 + 2 i2 + 4 i3) at position
// (sx + i1) + 3 (sy + i2) + 9 (sz + i3) of the 3 x 3 x 3 block.  A window of eight consecutive cells is an
// octant iff their entries agree wherever two of them meet one position (eight cells in Morton order
// form such a block only when they are the children of one octant, so the windows that pass do not
// overlap).
__device__ __forceinline__ int q1_octant_pos(int c, int n) {
  return ((c & 1) + (n & 1)) + 3 * (((c >> 1) & 1) + ((n >> 1) & 1)) + 9 * ((c >> 2) + (n >> 2));
}

// The 27 entries of the window starting at cell i, and whether it is an octant.
__device__ __forceinline__ bool q1_window(const int32_t* __restrict__ cell_dofs, int64_t i, int32_t (&e)[27]) {
#pragma unroll
  for (int p = 0; p < 27; ++p) e[p] = INT_MIN;
  bool ok = true;
  for (int c = 0; c < 8 && ok; ++c)
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const int32_t v = __ldg(cell_dofs + (i + c) * 8 + n);
      const int p = q1_octant_pos(c, n);
#pragma unroll
      for (int q = 0; q < 27; ++q)  // a compile-time-indexed register array: the slot by comparison
        if (q == p) {
          if (e[q] == INT_MIN) e[q] = v;
          else if (e[q] != v) ok = false;
        }
    }
  return ok;
}

__global__ void q1_window_kernel(int64_t n_cells, const int32_t* __restrict__ cell_dofs, uint8_t* __restrict__ pass) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_cells; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t e[27];
    pass[i] = (i + 8 <= n_cells && q1_window(cell_dofs, i, e)) ? 1 : 0;
  }
}

__global__ void q1_octant_dofs_kernel(int64_t n_oct, const int32_t* __restrict__ start,
                                      const int32_t* __restrict__ cell_dofs, int32_t* __restrict__ oct_dofs) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_oct; o += (int64_t)gridDim.x * blockDim.x) {
    int32_t e[27];
    q1_window(cell_dofs, start[o], e);
#pragma unroll
    for (int p = 0; p < 27; ++p) oct_dofs[o * 27 + p] = e[p];
  }
}

struct OctreeQ1Args {
  const int32_t* cell_dofs;  // n_cells x 8
  const int32_t* oct_start;  // first cell of each octant
  const int32_t* oct_dofs;   // per octant, its 27 node entries
  const int32_t* single;     // the cells outside octants
  int64_t n_oct, n_single;
  const int64_t* cptr;
  const int32_t* cmaster;
  const float* cweight;
  const float* box;  // [cell][3]: the metric diagonal over the quadrature weight
  float wq[2];       // Gauss weights
  const int32_t* skip;
};

// y = the Q1 cell operator applied to u (nodes i + 2 j + 4 l), metric w_q diag(D): gradients at the eight
// Gauss points by 1D contractions, the metric, the transposed contractions.
__device__ __forceinline__ void q1_cell_apply(const float (&u)[8], float wx0, float wx1, float D0, float D1, float D2,
                                              float (&y)[8]) {
  constexpr float S00 = (float)basis_entry<2, MAT_S>(0), S01 = (float)basis_entry<2, MAT_S>(1);
  constexpr float S10 = (float)basis_entry<2, MAT_S>(2), S11 = (float)basis_entry<2, MAT_S>(3);
  constexpr float T00 = (float)basis_entry<2, MAT_SD>(0), T01 = (float)basis_entry<2, MAT_SD>(1);
  constexpr float T10 = (float)basis_entry<2, MAT_SD>(2), T11 = (float)basis_entry<2, MAT_SD>(3);
  const float S[2][2] = {{S00, S01}, {S10, S11}}, T[2][2] = {{T00, T01}, {T10, T11}};
  const float w[2] = {wx0, wx1};
  // x: a = S_x u, b = Sd_x u, indexed [l][j][q]
  float a[2][2][2], b[2][2][2];
#pragma unroll
  for (int l = 0; l < 2; ++l)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        a[l][j][q] = S[q][0] * u[2 * j + 4 * l] + S[q][1] * u[1 + 2 * j + 4 * l];
        b[l][j][q] = T[q][0] * u[2 * j + 4 * l] + T[q][1] * u[1 + 2 * j + 4 * l];
      }
  // y: aa = S_y a, ab = Sd_y a, ba = S_y b, indexed [l][qy][qx]
  float aa[2][2][2], ab[2][2][2], ba[2][2][2];
#pragma unroll
  for (int l = 0; l < 2; ++l)
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        aa[l][p][q] = S[p][0] * a[l][0][q] + S[p][1] * a[l][1][q];
        ab[l][p][q] = T[p][0] * a[l][0][q] + T[p][1] * a[l][1][q];
        ba[l][p][q] = S[p][0] * b[l][0][q] + S[p][1] * b[l][1][q];
      }
  // z and the metric: h = w_q diag(D) (d/dx, d/dy, d/dz), indexed [qz][qy][qx]
  float hx[2][2][2], hy[2][2][2], hz[2][2][2];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const float wq = w[r] * w[p] * w[q];
        hx[r][p][q] = wq * D0 * (S[r][0] * ba[0][p][q] + S[r][1] * ba[1][p][q]);
        hy[r][p][q] = wq * D1 * (S[r][0] * ab[0][p][q] + S[r][1] * ab[1][p][q]);
        hz[r][p][q] = wq * D2 * (T[r][0] * aa[0][p][q] + T[r][1] * aa[1][p][q]);
      }
  // z^T: X = S_z^T hx, Y = S_z^T hy, Z = Sd_z^T hz, indexed [l][qy][qx]
  float X[2][2][2], Y[2][2][2], Z[2][2][2];
#pragma unroll
  for (int l = 0; l < 2; ++l)
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        X[l][p][q] = S[0][l] * hx[0][p][q] + S[1][l] * hx[1][p][q];
        Y[l][p][q] = S[0][l] * hy[0][p][q] + S[1][l] * hy[1][p][q];
        Z[l][p][q] = T[0][l] * hz[0][p][q] + T[1][l] * hz[1][p][q];
      }
  // y^T: A = S_y^T X (then Sd_x^T), B = Sd_y^T Y + S_y^T Z (then S_x^T), indexed [l][j][qx]
  float A[2][2][2], B[2][2][2];
#pragma unroll
  for (int l = 0; l < 2; ++l)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        A[l][j][q] = S[0][j] * X[l][0][q] + S[1][j] * X[l][1][q];
        B[l][j][q] = T[0][j] * Y[l][0][q] + T[1][j] * Y[l][1][q] + S[0][j] * Z[l][0][q] + S[1][j] * Z[l][1][q];
      }
  // x^T
#pragma unroll
  for (int l = 0; l < 2; ++l)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int i = 0; i < 2; ++i)
        y[i + 2 * j + 4 * l] =
            T[0][i] * A[l][j][0] + T[1][i] * A[l][j][1] + S[0][i] * B[l][j][0] + S[1][i] * B[l][j][1];
}

// Octants: a warp takes four (lane 8 g + c the child c of octant g), with the octants' 27 gathered values
// and 27 accumulated results in shared memory.
__global__ void __launch_bounds__(256) octree_q1_octant_kernel(const __grid_constant__ OctreeQ1Args a,
                                                                const float* __restrict__ src,
                                                                float* __restrict__ dst) {
  if (a.skip && *a.skip) return;
  __shared__ float vals[8][4][28], outs[8][4][28];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gi = lane >> 3, c8 = lane & 7;
  const int64_t n_wg = (a.n_oct + 3) / 4;
  for (int64_t wg = (int64_t)blockIdx.x * 8 + warp; wg < n_wg; wg += (int64_t)gridDim.x * 8) {
    const int64_t o = wg * 4 + gi;
    const bool act = o < a.n_oct;
    if (act)
      for (int t = c8; t < 27; t += 8) {
        vals[warp][gi][t] = gather_node(__ldg(a.oct_dofs + o * 27 + t), src, a.cptr, a.cmaster, a.cweight);
        outs[warp][gi][t] = 0.f;
      }
    __syncwarp();
    if (act) {
      const int64_t cell = __ldg(a.oct_start + o) + c8;
      float u[8], y[8];
#pragma unroll
      for (int n = 0; n < 8; ++n) u[n] = vals[warp][gi][q1_octant_pos(c8, n)];
      const float* Db = a.box + cell * 3;
      q1_cell_apply(u, a.wq[0], a.wq[1], __ldg(Db), __ldg(Db + 1), __ldg(Db + 2), y);
#pragma unroll
      for (int n = 0; n < 8; ++n) atomicAdd(&outs[warp][gi][q1_octant_pos(c8, n)], y[n]);
    }
    __syncwarp();
    if (act)
      for (int t = c8; t < 27; t += 8)
        scatter_node(__ldg(a.oct_dofs + o * 27 + t), outs[warp][gi][t], dst, a.cptr, a.cmaster, a.cweight);
    __syncwarp();
  }
}

// The cells outside octants: one thread per cell, gather and scatter per node.
__global__ void __launch_bounds__(256) octree_q1_single_kernel(const __grid_constant__ OctreeQ1Args a,
                                                               const float* __restrict__ src,
                                                               float* __restrict__ dst) {
  if (a.skip && *a.skip) return;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < a.n_single;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = __ldg(a.single + j);
    const int4 e0 = __ldg(reinterpret_cast<const int4*>(a.cell_dofs + cell * 8));
    const int4 e1 = __ldg(reinterpret_cast<const int4*>(a.cell_dofs + cell * 8 + 4));
    const int32_t e[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
    float u[8], y[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) u[n] = gather_node(e[n], src, a.cptr, a.cmaster, a.cweight);
    const float* Db = a.box + cell * 3;
    q1_cell_apply(u, a.wq[0], a.wq[1], __ldg(Db), __ldg(Db + 1), __ldg(Db + 2), y);
#pragma unroll
    for (int n = 0; n < 8; ++n) scatter_node(e[n], y[n], dst, a.cptr, a.cmaster, a.cweight);
  }
}

}  // namespace mfx
