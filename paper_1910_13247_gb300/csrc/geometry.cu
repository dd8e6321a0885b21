// Setup kernels: quadrature-point geometry (FP64), right-hand side,
// diagonal and constraint distribution.
//
// Geometry (Sec. 3.4: mapping + quadrature; Sec. 3.6: what to precompute):
// for every cell and Gauss point xi_q the trilinear map x(xi) of the cell's
// eight vertices gives J = dx/dxi, det J and J^-1; with the coefficient at
// the physical point the operator needs only the symmetric matrix
//     G_q = a(x_q) |det J_q| w_q J_q^-1 J_q^-T
// (six entries), stored per cell as [6][n^3] in FP64 and FP32.
#include <algorithm>
#include <cmath>

#include "mfx_internal.h"

namespace mfx {

struct GeoArgs {
  double xq[kMaxN], wq[kMaxN];
  double S[kMaxN * kMaxN], Sd[kMaxN * kMaxN];
  int n, k;
  int64_t n_cells;
  bool structured;
  int nx, ny, nz;
  const double* vertices;  // the (coarse) vertex lattice
  const int32_t* leaves;   // octree: (level, i, j, l) per cell
  int coef_kind;
  double par0, par1;
  const double* coef_q;
  int cb, nchunk;  // metric layout: cb = 0 -> [cell][6][q]; else [batch][6][q][cb] (structured rows)
  int cb32;        // FP32 copy: as cb (structured); octree: 0, or [cell / cb32][6][q][cb32] (runs of cells)
  bool runs32;     // FP32 copy of a structured mesh in the octree layouts (per cell, or runs of cb32 cells)
};

// Offset of metric entry (cell, 0, q) in the layout of batch size cb; entry e is at
// offset + e * metric_stride_cb(g, cb).
__device__ __forceinline__ int64_t metric_offset_cb(const GeoArgs& g, int64_t cell, int q, int cb) {
  const int n3 = g.n * g.n * g.n;
  if (cb == 0) return cell * 6 * n3 + q;
  if (!g.structured) {
    const int64_t batch = cell / cb;
    return (batch * 6 * n3 + q) * cb + (cell - batch * cb);
  }
  const int cx = (int)(cell % g.nx);
  const int64_t rest = cell / g.nx;
  const int cy = (int)(rest % g.ny), cz = (int)(rest / g.ny);
  const int chunk = cx / cb, c = cx - chunk * cb;
  const int64_t batch = chunk + (int64_t)g.nchunk * (cy + (int64_t)g.ny * cz);
  return (batch * 6 * n3 + q) * cb + c;
}
__device__ __forceinline__ int64_t metric_stride_cb(const GeoArgs& g, int cb) {
  const int n3 = g.n * g.n * g.n;
  return cb == 0 ? (int64_t)n3 : (int64_t)n3 * cb;
}
// The FP64 metric's layout.
__device__ __forceinline__ int64_t metric_offset(const GeoArgs& g, int64_t cell, int q) {
  return metric_offset_cb(g, cell, q, g.cb);
}
__device__ __forceinline__ int64_t metric_stride(const GeoArgs& g) { return metric_stride_cb(g, g.cb); }

__device__ __forceinline__ void cell_vertices(const GeoArgs& g, int64_t cell, double V[8][3]) {
  if (g.structured) {
    const int cx = (int)(cell % g.nx);
    const int64_t rest = cell / g.nx;
    const int cy = (int)(rest % g.ny), cz = (int)(rest / g.ny);
    for (int v = 0; v < 8; ++v) {
      const int a = v & 1, b = (v >> 1) & 1, c = (v >> 2) & 1;
      const int64_t idx = (cx + a) + (int64_t)(g.nx + 1) * ((cy + b) + (int64_t)(g.ny + 1) * (cz + c));
      for (int d = 0; d < 3; ++d) V[v][d] = g.vertices[3 * idx + d];
    }
  } else {
    // the leaf's corners: the trilinear map of its coarse cell at the reference points (I + a) / 2^L
    const int L = g.leaves[4 * cell], li = g.leaves[4 * cell + 1], lj = g.leaves[4 * cell + 2],
              ll = g.leaves[4 * cell + 3];
    const int ci = li >> L, cj = lj >> L, cl = ll >> L;
    double X[8][3];
    for (int w = 0; w < 8; ++w) {
      const int a = w & 1, b = (w >> 1) & 1, c = (w >> 2) & 1;
      const int64_t idx = (ci + a) + (int64_t)(g.nx + 1) * ((cj + b) + (int64_t)(g.ny + 1) * (cl + c));
      for (int d = 0; d < 3; ++d) X[w][d] = g.vertices[3 * idx + d];
    }
    const double h = 1.0 / (double)(1 << L);
    for (int v = 0; v < 8; ++v) {
      const double s = (double)(li - (ci << L) + (v & 1)) * h;
      const double t = (double)(lj - (cj << L) + ((v >> 1) & 1)) * h;
      const double u = (double)(ll - (cl << L) + ((v >> 2) & 1)) * h;
      for (int d = 0; d < 3; ++d) {
        double p = 0.0;
        for (int w = 0; w < 8; ++w)
          p += ((w & 1) ? s : 1.0 - s) * ((w & 2) ? t : 1.0 - t) * ((w & 4) ? u : 1.0 - u) * X[w][d];
        V[v][d] = p;
      }
    }
  }
}

// Trilinear map at reference point xi: x and J[i][j] = dx_i / dxi_j.
__device__ __forceinline__ void q1_map(const double V[8][3], const double xi[3], double x[3], double J[3][3]) {
  for (int i = 0; i < 3; ++i) {
    x[i] = 0.0;
    for (int j = 0; j < 3; ++j) J[i][j] = 0.0;
  }
  for (int v = 0; v < 8; ++v) {
    const int c[3] = {v & 1, (v >> 1) & 1, (v >> 2) & 1};
    double N[3], dN[3];
    for (int d = 0; d < 3; ++d) {
      N[d] = c[d] ? xi[d] : 1.0 - xi[d];
      dN[d] = c[d] ? 1.0 : -1.0;
    }
    const double sh = N[0] * N[1] * N[2];
    const double gr[3] = {dN[0] * N[1] * N[2], N[0] * dN[1] * N[2], N[0] * N[1] * dN[2]};
    for (int i = 0; i < 3; ++i) {
      x[i] += sh * V[v][i];
      for (int j = 0; j < 3; ++j) J[i][j] += V[v][i] * gr[j];
    }
  }
}

__device__ __forceinline__ double invert3(const double J[3][3], double Ji[3][3]) {
  const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  const double id = 1.0 / det;
  Ji[0][0] = c00 * id;
  Ji[1][0] = c01 * id;
  Ji[2][0] = c02 * id;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
  return det;
}

__global__ void geometry_kernel(const __grid_constant__ GeoArgs g, double* __restrict__ m64,
                                float* __restrict__ m32, double* __restrict__ jxw) {
  const int n = g.n, n3 = n * n * n;
  const int64_t total = g.n_cells * n3;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = idx / n3;
    const int q = (int)(idx - cell * n3);
    const int q1 = q % n, q2 = (q / n) % n, q3 = q / (n * n);
    double V[8][3];
    cell_vertices(g, cell, V);
    const double xi[3] = {g.xq[q1], g.xq[q2], g.xq[q3]};
    double x[3], J[3][3], Ji[3][3];
    q1_map(V, xi, x, J);
    const double det = invert3(J, Ji);
    double a;
    if (g.coef_kind == MFX_COEF_CONSTANT)
      a = g.par0;
    else if (g.coef_kind == MFX_COEF_TRIG)
      a = g.par0 + g.par1 * sinpi(2.0 * x[0]) * cospi(2.0 * x[1]) * x[2];
    else
      a = g.coef_q[idx];
    const double w = g.wq[q1] * g.wq[q2] * g.wq[q3];
    const double dx = fabs(det) * w;
    const double f = a * dx;
    double G[6];
    const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
    for (int e = 0; e < 6; ++e) {
      const int r = ia[e], c = ib[e];
      G[e] = f * (Ji[r][0] * Ji[c][0] + Ji[r][1] * Ji[c][1] + Ji[r][2] * Ji[c][2]);
    }
    const int64_t base = metric_offset(g, cell, q), st = metric_stride(g);
    int64_t base32;
    if (g.runs32 && g.cb32 > 0) {  // runs of cb32 consecutive cells
      const int64_t batch = cell / g.cb32;
      base32 = (batch * 6 * (int64_t)g.n * g.n * g.n + q) * g.cb32 + (cell - batch * g.cb32);
    } else {
      base32 = metric_offset_cb(g, cell, q, g.cb32);
    }
    const int64_t st32 = metric_stride_cb(g, g.cb32);
    for (int e = 0; e < 6; ++e) {
      if (m64) m64[base + e * st] = G[e];
      if (m32) m32[base32 + e * st32] = (float)G[e];
    }
    if (jxw) jxw[idx] = dx;
  }
}

__global__ void qpoints_kernel(const __grid_constant__ GeoArgs g, double* __restrict__ out) {
  const int n = g.n, n3 = n * n * n;
  const int64_t total = g.n_cells * n3;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = idx / n3;
    const int q = (int)(idx - cell * n3);
    double V[8][3];
    cell_vertices(g, cell, V);
    const double xi[3] = {g.xq[q % n], g.xq[(q / n) % n], g.xq[q / (n * n)]};
    double x[3], J[3][3];
    q1_map(V, xi, x, J);
    for (int d = 0; d < 3; ++d) out[3 * idx + d] = x[d];
  }
}

// Global DoF of local node (i1, i2, i3) and its constraint class.
struct DofView {
  bool structured;
  uint32_t dmask;  // structured: Dirichlet faces
  int nx, ny, k, Mx, My, Mz, n;
  const int32_t* cell_dofs;
  const int64_t* cptr;
  const int32_t* cmaster;
  const double* cweight;
};

// Calls f(dof, weight) for every free DoF the local node expands to.
template <typename F>
__device__ __forceinline__ void expand_node(const DofView& v, int64_t cell, int i1, int i2, int i3, F f) {
  if (v.structured) {
    const int cx = (int)(cell % v.nx);
    const int64_t rest = cell / v.nx;
    const int cy = (int)(rest % v.ny), cz = (int)(rest / v.ny);
    const int I = cx * v.k + i1, J = cy * v.k + i2, L = cz * v.k + i3;
    if (on_dirichlet(v.dmask, I, J, L, v.Mx, v.My, v.Mz)) return;
    f((int64_t)I + (int64_t)v.Mx * (J + (int64_t)v.My * L), 1.0);
  } else {
    const int32_t e = v.cell_dofs[cell * v.n * v.n * v.n + (i3 * v.n + i2) * v.n + i1];
    if (e >= 0) {
      f((int64_t)e, 1.0);
    } else {
      const int32_t row = -e - 1;
      for (int64_t p = v.cptr[row]; p < v.cptr[row + 1]; ++p) f((int64_t)v.cmaster[p], v.cweight[p]);
    }
  }
}

__global__ void rhs_kernel(const __grid_constant__ GeoArgs g, DofView v, const double* __restrict__ fq,
                           const double* __restrict__ jxw, double* __restrict__ b) {
  const int n = g.n, n3 = n * n * n;
  const int64_t total = g.n_cells * n3;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = idx / n3;
    const int i = (int)(idx - cell * n3);
    const int i1 = i % n, i2 = (i / n) % n, i3 = i / (n * n);
    double s = 0.0;
    for (int q = 0; q < n3; ++q) {
      const int q1 = q % n, q2 = (q / n) % n, q3 = q / (n * n);
      const double phi = g.S[q1 * n + i1] * g.S[q2 * n + i2] * g.S[q3 * n + i3];
      s += phi * fq[cell * n3 + q] * jxw[cell * n3 + q];
    }
    expand_node(v, cell, i1, i2, i3, [&](int64_t dof, double w) { atomicAdd(b + dof, w * s); });
  }
}

// Diagonal of the element matrices by sum factorisation.  With the 1D
// products M0[q][i] = l_i(x_q)^2, M1[q][i] = l_i(x_q) l_i'(x_q), M2[q][i] = l_i'(x_q)^2, the entry
// A_ii of node i = (i1, i2, i3) is the sum over the six metric components G_de of
//   c_de sum_q G_de(q) M_{a1}[q1][i1] M_{a2}[q2][i2] M_{a3}[q3][i3],
// a_t = [t == d] + [t == e], c_de = 1 for d = e and 2 otherwise (G symmetric): three 1D contractions
// (over q3, q2, q1) per component instead of n^3 quadrature sums per node.  N^2 threads per cell,
// one per 1D line; CPB cells per CTA.  On a cell with hanging nodes only the nodes flagged in
// `simple` (free DoFs that no hanging node of the cell depends on) are added here; the other shares
// come from diagonal_hanging_kernel.
template <int N>
__global__ void diagonal_sf_kernel(const __grid_constant__ GeoArgs g, DofView v, const double* __restrict__ m64,
                                   const uint8_t* __restrict__ cell_hanging, const uint8_t* __restrict__ simple,
                                   double* __restrict__ diag, int cpb) {
  constexpr int N2 = N * N, N3 = N2 * N;
  extern __shared__ double sh[];
  double* M = sh;  // 3 x N^2
  const int lc = threadIdx.x / N2;
  const int r = threadIdx.x - lc * N2;
  double* X = sh + 3 * N2 + lc * 2 * N3;
  double* Y = X + N3;
  for (int t = threadIdx.x; t < N2; t += blockDim.x) {
    const double s0 = g.S[t], s1 = g.Sd[t];
    M[t] = s0 * s0;
    M[N2 + t] = s0 * s1;
    M[2 * N2 + t] = s1 * s1;
  }
  const int64_t cell = (int64_t)blockIdx.x * cpb + lc;
  const bool ok = lc < cpb && cell < g.n_cells;
  const bool hang = ok && cell_hanging && cell_hanging[cell];
  const int64_t base = ok ? metric_offset(g, cell, 0) : 0;
  const int64_t st = metric_stride(g);
  const int ra = r % N, rb = r / N;
  double z[N];
#pragma unroll
  for (int i = 0; i < N; ++i) z[i] = 0.0;
  __syncthreads();
#pragma unroll 1
  for (int c = 0; c < 6; ++c) {  // components G00, G01, G02, G11, G12, G22
    const int d = c < 3 ? 0 : (c < 5 ? 1 : 2);
    const int e = c < 3 ? c : (c < 5 ? c - 2 : 2);
    const double* T1 = M + ((d == 0) + (e == 0)) * N2;
    const double* T2 = M + ((d == 1) + (e == 1)) * N2;
    const double* T3 = M + ((d == 2) + (e == 2)) * N2;
    // contraction over q3: thread (q1, q2) = (ra, rb)
    if (ok) {
      double gq[N];
#pragma unroll
      for (int q3 = 0; q3 < N; ++q3) {
        const int q = ra + N * rb + N2 * q3;
        gq[q3] = m64[base + c * st + (g.cb == 0 ? q : (int64_t)q * g.cb)];
      }
#pragma unroll
      for (int i3 = 0; i3 < N; ++i3) {
        double acc = 0.0;
#pragma unroll
        for (int q3 = 0; q3 < N; ++q3) acc += gq[q3] * T3[q3 * N + i3];
        X[ra + N * rb + N2 * i3] = acc;
      }
    }
    __syncthreads();
    // contraction over q2: thread (q1, i3) = (ra, rb)
    if (ok) {
#pragma unroll
      for (int i2 = 0; i2 < N; ++i2) {
        double acc = 0.0;
#pragma unroll
        for (int q2 = 0; q2 < N; ++q2) acc += X[ra + N * q2 + N2 * rb] * T2[q2 * N + i2];
        Y[ra + N * i2 + N2 * rb] = acc;
      }
    }
    __syncthreads();
    // contraction over q1: thread (i2, i3) = (ra, rb)
    if (ok) {
      const double cde = d == e ? 1.0 : 2.0;
#pragma unroll
      for (int i1 = 0; i1 < N; ++i1) {
        double acc = 0.0;
#pragma unroll
        for (int q1 = 0; q1 < N; ++q1) acc += Y[q1 + N * ra + N2 * rb] * T1[q1 * N + i1];
        z[i1] += cde * acc;
      }
    }
    __syncthreads();
  }
  if (ok) {
#pragma unroll
    for (int i1 = 0; i1 < N; ++i1) {
      if (hang && !simple[cell * N3 + i1 + N * ra + N2 * rb]) continue;
      expand_node(v, cell, i1, ra, rb, [&](int64_t dof, double w) { atomicAdd(diag + dof, w * w * z[i1]); });
    }
  }
}

// One 1D sweep of an n^3 array along direction dir (0: x = i1, 1: y = i2, 2: z = i3) with the
// matrix M[q][i]; thread t owns the line whose other two indices are (t mod N, t / N).
template <int N>
__device__ __forceinline__ void sweep3(const double* in, double* out, const double* M, int dir, int t) {
  constexpr int N2 = N * N;
  const int a = t % N, b = t / N;
  const int base = dir == 0 ? N * a + N2 * b : (dir == 1 ? a + N2 * b : a + N * b);
  const int stride = dir == 0 ? 1 : (dir == 1 ? N : N2);
  double x[N];
#pragma unroll
  for (int i = 0; i < N; ++i) x[i] = in[base + i * stride];
#pragma unroll
  for (int q = 0; q < N; ++q) {
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) acc += M[q * N + i] * x[i];
    out[base + q * stride] = acc;
  }
}

// Share of master m in diag(C^T A C) from one cell with hanging nodes: with v the m-th column of the
// cell's constraint matrix (v_i = 1 where node i is the free DoF m, the weight of m where node i is
// hanging, else 0), the share is v^T A_cell v = sum_q grad v(q)^T G_q grad v(q).  The reference
// gradient at the Gauss points takes eight sum-factorisation sweeps in three phases:
//   S_z v, D_z v  ->  S_y S_z v, D_y S_z v, S_y D_z v  ->  D_x S_y S_z v, S_x D_y S_z v, S_x S_y D_z v.
// One CTA of N^2 threads (one per 1D line) per (cell, master) job.
template <int N>
__global__ void diagonal_hanging_kernel(const __grid_constant__ GeoArgs g, DofView dv, const double* __restrict__ m64,
                                        const int32_t* __restrict__ job_cell, const int32_t* __restrict__ job_master,
                                        double* __restrict__ diag) {
  constexpr int N2 = N * N, N3 = N2 * N;
  __shared__ double S[N2], Sd[N2], red[N2];
  __shared__ double v[N3], A[N3], B[N3], C[N3], D[N3], E[N3];
  const int t = threadIdx.x;
  const int64_t cell = job_cell[blockIdx.x];
  const int32_t m = job_master[blockIdx.x];
  S[t] = g.S[t];
  Sd[t] = g.Sd[t];
  for (int i = t; i < N3; i += N2) {
    const int32_t e = dv.cell_dofs[cell * N3 + i];
    double w = 0.0;
    if (e >= 0) {
      w = e == m ? 1.0 : 0.0;
    } else {
      const int32_t row = -e - 1;
      for (int64_t p = dv.cptr[row]; p < dv.cptr[row + 1]; ++p)
        if (dv.cmaster[p] == m) w += dv.cweight[p];
    }
    v[i] = w;
  }
  __syncthreads();
  sweep3<N>(v, A, S, 2, t);   // A = S_z v
  sweep3<N>(v, B, Sd, 2, t);  // B = D_z v
  __syncthreads();
  sweep3<N>(A, C, S, 1, t);   // C = S_y S_z v
  sweep3<N>(A, D, Sd, 1, t);  // D = D_y S_z v
  sweep3<N>(B, E, S, 1, t);   // E = S_y D_z v
  __syncthreads();
  sweep3<N>(C, v, Sd, 0, t);  // grad_x -> v
  sweep3<N>(D, A, S, 0, t);   // grad_y -> A
  sweep3<N>(E, B, S, 0, t);   // grad_z -> B
  __syncthreads();
  const int64_t base = metric_offset(g, cell, 0), st = metric_stride(g);
  const int64_t qs = g.cb == 0 ? 1 : g.cb;
  double acc = 0.0;
  for (int q = t; q < N3; q += N2) {
    const double* G = m64 + base + q * qs;
    const double u1 = v[q], u2 = A[q], u3 = B[q];
    acc += u1 * (G[0] * u1 + 2.0 * (G[st] * u2 + G[2 * st] * u3)) + u2 * (G[3 * st] * u2 + 2.0 * G[4 * st] * u3) +
           u3 * G[5 * st] * u3;
  }
  red[t] = acc;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int w = 0; w < N2; ++w) s += red[w];
    atomicAdd(diag + m, s);
  }
}

template <typename Real>
__global__ void diag_finish_kernel(int64_t n_dofs, bool structured, uint32_t dmask, int Mx, int My, int Mz,
                                   const uint8_t* __restrict__ cmask, const double* __restrict__ d,
                                   double* __restrict__ d64, float* __restrict__ d32) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_dofs; i += (int64_t)gridDim.x * blockDim.x) {
    bool c;
    if (structured) {
      const int64_t I = i % Mx, rest = i / Mx, J = rest % My, L = rest / My;
      c = on_dirichlet(dmask, I, J, L, Mx, My, Mz);
    } else {
      c = cmask[i] != 0;
    }
    const double val = c ? 1.0 : d[i];
    if (d64) d64[i] = val;
    if (d32) d32[i] = (float)val;
  }
}

__global__ void distribute_kernel(int64_t n_dofs, bool structured, uint32_t dmask, int Mx, int My, int Mz,
                                  int64_t n_constrained,
                                  const int32_t* __restrict__ constrained, const int64_t* __restrict__ cptr,
                                  const int32_t* __restrict__ cmaster, const double* __restrict__ cweight,
                                  double* __restrict__ x) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (structured) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_dofs; i += stride) {
      const int64_t I = i % Mx, rest = i / Mx, J = rest % My, L = rest / My;
      if (on_dirichlet(dmask, I, J, L, Mx, My, Mz)) x[i] = 0.0;
    }
    return;
  }
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_constrained; t += stride) {
    double s = 0.0;
    for (int64_t p = cptr[t]; p < cptr[t + 1]; ++p) s += cweight[p] * x[cmaster[p]];
    x[constrained[t]] = s;
  }
}

static GeoArgs geo_args(const mfx_op* op) {
  GeoArgs g;
  const int n = op->n;
  for (int i = 0; i < n; ++i) {
    g.xq[i] = op->basis.xq[i];
    g.wq[i] = op->basis.wq[i];
  }
  for (int i = 0; i < n * n; ++i) {
    g.S[i] = op->basis.S[i];
    g.Sd[i] = op->basis.Sd[i];
  }
  g.n = n;
  g.k = op->k;
  g.n_cells = op->n_cells;
  g.structured = op->structured;
  g.nx = op->nx;
  g.ny = op->ny;
  g.nz = op->nz;
  g.vertices = op->d_vertices;
  g.leaves = op->d_leaves;
  g.coef_kind = MFX_COEF_CONSTANT;
  g.par0 = 1.0;
  g.par1 = 0.0;
  g.coef_q = nullptr;
  g.cb = op->metric_cb;
  g.nchunk = op->nchunk;
  g.cb32 = op->structured && !op->percell32 ? op->metric_cb : op->metric_cb32;
  g.runs32 = op->percell32;
  return g;
}

// Index tables of a structured mesh for the per-cell kernels: lattice index of every cell node, -1 on
// Dirichlet points (a constraint row without masters), and the per-DoF constrained mask.
__global__ void structured_cell_dofs_kernel(int64_t n_cells, int nx, int ny, int n, int Mx, int My, int Mz,
                                            uint32_t dmask, int32_t* __restrict__ cell_dofs) {
  const int n3 = n * n * n, k = n - 1;
  const int64_t total = n_cells * n3;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = idx / n3;
    const int i = (int)(idx - cell * n3);
    const int64_t I = (cell % nx) * k + i % n, J = ((cell / nx) % ny) * k + (i / n) % n,
                  L = (cell / ((int64_t)nx * ny)) * k + i / (n * n);
    cell_dofs[idx] = on_dirichlet(dmask, I, J, L, Mx, My, Mz) ? -1 : (int32_t)(I + (int64_t)Mx * (J + (int64_t)My * L));
  }
}
__global__ void structured_cmask_kernel(int Mx, int My, int Mz, uint32_t dmask, uint8_t* __restrict__ mask) {
  const int64_t total = (int64_t)Mx * My * Mz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = i % Mx, rest = i / Mx, J = rest % My, L = rest / My;
    mask[i] = on_dirichlet(dmask, I, J, L, Mx, My, Mz) ? 1 : 0;
  }
}

static int grid_for(int64_t work);

mfx_status launch_structured_index_tables(mfx_op* op, cudaStream_t s) {
  const int Mx = op->k * op->nx + 1, My = op->k * op->ny + 1, Mz = op->k * op->nz + 1;
  const int64_t work = op->n_cells * op->n * op->n * op->n;
  structured_cell_dofs_kernel<<<grid_for(work), 256, 0, s>>>(op->n_cells, op->nx, op->ny, op->n, Mx, My, Mz,
                                                              op->dirichlet, op->d_cell_dofs);
  structured_cmask_kernel<<<grid_for(op->n_dofs), 256, 0, s>>>(Mx, My, Mz, op->dirichlet, op->d_cmask);
  MFX_CUDA_TRY(cudaMemsetAsync(op->d_cptr, 0, 2 * sizeof(int64_t), s));
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

static DofView dof_view(const mfx_op* op) {
  DofView v;
  v.structured = op->structured;
  v.dmask = op->dirichlet;
  v.nx = op->nx;
  v.ny = op->ny;
  v.k = op->k;
  v.Mx = op->k * op->nx + 1;
  v.My = op->k * op->ny + 1;
  v.Mz = op->k * op->nz + 1;
  v.n = op->n;
  v.cell_dofs = op->d_cell_dofs;
  v.cptr = op->d_cptr;
  v.cmaster = op->d_cmaster;
  v.cweight = op->d_cweight64;
  return v;
}

static int grid_for(int64_t work) {
  const int64_t b = (work + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)device_sm_count() * 16));
}

mfx_status launch_geometry(mfx_op* op, int coef_kind, const double* par, const double* coef_q, cudaStream_t s) {
  GeoArgs g = geo_args(op);
  g.coef_kind = coef_kind;
  g.par0 = par[0];
  g.par1 = par[1];
  g.coef_q = coef_q;
  const int64_t work = op->n_cells * op->n * op->n * op->n;
  geometry_kernel<<<grid_for(work), 256, 0, s>>>(g, op->d_metric64, op->d_metric32, op->d_jxw);
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

mfx_status launch_qpoints(const mfx_op* op, double* xq, cudaStream_t s) {
  if (op->dg) return launch_dg_qpoints(op, xq, s);
  GeoArgs g = geo_args(op);
  const int64_t work = op->n_cells * op->n * op->n * op->n;
  qpoints_kernel<<<grid_for(work), 256, 0, s>>>(g, xq);
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

mfx_status launch_rhs(const mfx_op* op, const double* fq, double* b, cudaStream_t s) {
  if (op->dg) return launch_dg_rhs(op, fq, b, s);
  GeoArgs g = geo_args(op);
  MFX_CUDA_TRY(cudaMemsetAsync(b, 0, sizeof(double) * op->n_dofs, s));
  const int64_t work = op->n_cells * op->n * op->n * op->n;
  rhs_kernel<<<grid_for(work), 256, 0, s>>>(g, dof_view(op), fq, op->d_jxw, b);
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

template <int N>
static void run_diagonal_sf(const GeoArgs& g, const DofView& v, const double* m64, const uint8_t* hang,
                            const uint8_t* simple, const int32_t* job_cell, const int32_t* job_master, int64_t n_jobs,
                            double* d, cudaStream_t s) {
  constexpr int cpb = N * N >= 64 ? 1 : 128 / (N * N);  // cells per CTA
  const int64_t blocks = (g.n_cells + cpb - 1) / cpb;
  if (blocks == 0) return;
  const size_t smem = sizeof(double) * (3 * N * N + 2 * cpb * N * N * N);
  diagonal_sf_kernel<N><<<(unsigned)blocks, cpb * N * N, smem, s>>>(g, v, m64, hang, simple, d, cpb);
  if (n_jobs > 0) diagonal_hanging_kernel<N><<<(unsigned)n_jobs, N * N, 0, s>>>(g, v, m64, job_cell, job_master, d);
}

static void launch_diagonal_sf(int n, const GeoArgs& g, const DofView& v, const double* m64, const uint8_t* hang,
                               const uint8_t* simple, const int32_t* jc, const int32_t* jm, int64_t nj, double* d,
                               cudaStream_t s) {
  switch (n) {
    case 2: run_diagonal_sf<2>(g, v, m64, hang, simple, jc, jm, nj, d, s); break;
    case 3: run_diagonal_sf<3>(g, v, m64, hang, simple, jc, jm, nj, d, s); break;
    case 4: run_diagonal_sf<4>(g, v, m64, hang, simple, jc, jm, nj, d, s); break;
    case 5: run_diagonal_sf<5>(g, v, m64, hang, simple, jc, jm, nj, d, s); break;
    case 6: run_diagonal_sf<6>(g, v, m64, hang, simple, jc, jm, nj, d, s); break;
    case 7: run_diagonal_sf<7>(g, v, m64, hang, simple, jc, jm, nj, d, s); break;
    case 8: run_diagonal_sf<8>(g, v, m64, hang, simple, jc, jm, nj, d, s); break;
    case 9: run_diagonal_sf<9>(g, v, m64, hang, simple, jc, jm, nj, d, s); break;
    default: break;
  }
}

mfx_status launch_diagonal(mfx_op* op, cudaStream_t s) {
  GeoArgs g = geo_args(op);
  double* tmp = nullptr;
  uint8_t* simple = nullptr;
  int32_t* jobs = nullptr;
  const int64_t nj = (int64_t)op->hang_job_cell.size();
  MFX_CUDA_TRY(cudaMallocAsync((void**)&tmp, sizeof(double) * std::max<int64_t>(1, op->n_dofs), s));
  cudaError_t e = cudaMemsetAsync(tmp, 0, sizeof(double) * op->n_dofs, s);
  if (e == cudaSuccess && op->d_cell_hanging && !op->hang_simple.empty()) {
    e = cudaMallocAsync((void**)&simple, op->hang_simple.size(), s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(simple, op->hang_simple.data(), op->hang_simple.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nj > 0) e = cudaMallocAsync((void**)&jobs, sizeof(int32_t) * 2 * nj, s);
    if (e == cudaSuccess && nj > 0)
      e = cudaMemcpyAsync(jobs, op->hang_job_cell.data(), sizeof(int32_t) * nj, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nj > 0)
      e = cudaMemcpyAsync(jobs + nj, op->hang_job_master.data(), sizeof(int32_t) * nj, cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) {
    launch_diagonal_sf(op->n, g, dof_view(op), op->d_metric64, simple ? op->d_cell_hanging : nullptr, simple, jobs,
                       jobs ? jobs + nj : nullptr, jobs ? nj : 0, tmp, s);
    diag_finish_kernel<double><<<grid_for(op->n_dofs), 256, 0, s>>>(
        op->n_dofs, op->structured, op->dirichlet, op->k * op->nx + 1, op->k * op->ny + 1, op->k * op->nz + 1, op->d_cmask, tmp,
        op->d_diag64, op->d_diag32);
    e = cudaGetLastError();
  }
  cudaFreeAsync(tmp, s);
  if (simple) cudaFreeAsync(simple, s);
  if (jobs) cudaFreeAsync(jobs, s);
  if (e != cudaSuccess) return cuda_error(e, "diagonal");
  return MFX_OK;
}

// Box cells (axis-aligned boxes with a constant coefficient): the metric at quadrature point q is
// w_q a |det J| J^-1 J^-T with a constant diagonal J, i.e. w_q diag(D).  One thread per cell: D from the
// first point, every point and entry checked against w_q diag(D) to 1e-12 of the largest entry of D.
__global__ void box_check_kernel(const GeoArgs g, const double* __restrict__ m64, float* __restrict__ box,
                                 int* __restrict__ not_box) {
  const int n = g.n, n3 = n * n * n;
  const int64_t st = metric_stride(g);
  for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < g.n_cells;
       cell += (int64_t)gridDim.x * blockDim.x) {
    const double w0 = g.wq[0] * g.wq[0] * g.wq[0];
    const int64_t b0 = metric_offset(g, cell, 0);
    const double D[3] = {m64[b0] / w0, m64[b0 + 3 * st] / w0, m64[b0 + 5 * st] / w0};
    const double tol = 1e-12 * fmax(fabs(D[0]), fmax(fabs(D[1]), fabs(D[2])));
    bool ok = true;
    for (int q = 0; q < n3 && ok; ++q) {
      const double w = g.wq[q % n] * g.wq[(q / n) % n] * g.wq[q / (n * n)];
      const int64_t b = metric_offset(g, cell, q);
      const double expect[6] = {D[0], 0.0, 0.0, D[1], 0.0, D[2]};
      for (int e = 0; e < 6; ++e) ok = ok && fabs(m64[b + e * st] / w - expect[e]) <= tol;
    }
    if (!ok) atomicOr(not_box, 1);
    for (int i = 0; i < 3; ++i) box[cell * 3 + i] = (float)D[i];
  }
}

mfx_status launch_box_check(const mfx_op* op, float* box, int* not_box, cudaStream_t s) {
  const GeoArgs g = geo_args(op);
  box_check_kernel<<<grid_for(op->n_cells), 256, 0, s>>>(g, op->d_metric64, box, not_box);
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

// FP64 metric -> (hi, lo) float pairs in place (structured operators, after the FP64 diagonal).
__global__ void metric_to_pairs_kernel(int64_t n, double* __restrict__ m) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = m[i];
    const float h = __double2float_rn(v);
    const float l = __double2float_rn(v - (double)h);
    reinterpret_cast<float2*>(m)[i] = make_float2(h, l);
  }
}

mfx_status launch_metric_to_pairs(mfx_op* op, int64_t entries, cudaStream_t s) {
  metric_to_pairs_kernel<<<grid_for(entries), 256, 0, s>>>(entries, op->d_metric64);
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

mfx_status launch_distribute(const mfx_op* op, double* x, cudaStream_t s) {
  const int64_t work = op->structured ? op->n_dofs : op->n_constrained;
  if (work == 0) return MFX_OK;
  distribute_kernel<<<grid_for(work), 256, 0, s>>>(op->n_dofs, op->structured, op->dirichlet, op->k * op->nx + 1,
                                                   op->k * op->ny + 1, op->k * op->nz + 1, op->n_constrained,
                                                   op->d_constrained, op->d_cptr, op->d_cmaster, op->d_cweight64, x);
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

}  // namespace mfx
