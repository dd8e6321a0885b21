// Matrix-free application of the Q_k Laplacian (Sec. 3.6), one degree per
// translation unit (MFX_N = k + 1 defined by the including file).
//
// Design (GB300):
//  * a CTA of 256 threads owns CB = floor(256 / n^2) cells at a time and
//    walks the cell range persistently (grid = resident CTAs on all SMs);
//  * every 1D contraction is done by a thread that owns one line of one
//    cell: it reads the n values of the line (from HBM in the gather, from
//    shared memory otherwise), applies the n x n matrix held in the kernel
//    parameter bank (uniform operands, no memory traffic) and writes the n
//    results back; the cell data lives in three shared-memory cubes per
//    cell, rows padded to an odd length so line accesses are conflict-free;
//  * the metric (6 values per quadrature point) is streamed from HBM once,
//    coalesced, by the thread that owns the z-line of quadrature points;
//  * the scatter adds the cell results with fire-and-forget atomics; the
//    constrained rows are written by a prologue kernel (identity rows).
//
// Steps per cell (n = k + 1 Gauss points per direction):
//   gather (+ constraints) -> S_x -> S_y -> S_z (values at Gauss points)
//   -> D_x, D_y, D_z (reference gradient, collocation derivative on the
//   Gauss points) -> h = G_q grad (G = a |det J| w J^-1 J^-T)
//   -> D_x^T h1 + D_y^T h2 + D_z^T h3 -> S_z^T -> S_y^T -> S_x^T -> scatter.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "basis_tables.h"

namespace mfx {

template <int N, typename Real>
struct VmultArgs {
  const Real* metric;  // [cell][6][N^3]
  int64_t n_cells;
  const int32_t* cell_dofs;  // >= 0 free DoF, < 0: -(row + 1) into the constraint rows
  const int64_t* cptr;
  const int32_t* cmaster;
  const Real* cweight;
  const uint8_t* cmask;
  int64_t n_dofs;
  const int32_t* skip;  // optional: when *skip != 0 the launch does nothing (converged solve)
  // optional (octree): hanging constraints in tensor-product form, per cell (see OctreeTables::hface):
  // a hanging face's constrained nodes are the coarse face's Q_k function at the fine nodes, two 1D
  // interpolations P[c][b][m] = l_m((c + x_b) / 2) (c the half of the coarse face the fine face covers);
  // a hanging edge's, one
  const uint32_t* hface;
  const uint32_t* hedge;
  const int64_t* hoff;
  const int32_t* hdofs;
  Real P[2 * N * N];
  // optional: the launch processes the cells cell_list[0 .. n_list) instead of 0 .. n_cells
  const int32_t* cell_list;
  int64_t n_list;
  // box cells (FP32 kernels built for them): the metric at quadrature point (q1, q2, q3) of a cell is
  // wq[q1] wq[q2] wq[q3] diag(box[cell][0..2])
  const float* box;
  Real wq[N];
};

// The hanging face (0..5) or edge (6..17) of a cell that owns local node (a1, a2, a3): the first hanging
// face containing it, else the first hanging edge, else -1.  Each constrained node of a cell with
// hanging faces or edges is interpolated by exactly one owner, and its transpose goes back through the
// same owner only.
// A node lies on at most one face and one edge per axis, found from its coordinates: face 2 d + side if
// a_d is 0 or K, edge 4 d + 2 side_v + side_u (u, v the lower and the higher of the other two axes) if
// a_u and a_v both are; the faces and then the edges are tried in ascending index order.
__device__ __forceinline__ int hang_owner(uint32_t hf, uint32_t he, int a1, int a2, int a3, int K) {
  const bool lo1 = a1 == 0, hi1 = a1 == K, lo2 = a2 == 0, hi2 = a2 == K, lo3 = a3 == 0, hi3 = a3 == K;
  const bool e1 = lo1 || hi1, e2 = lo2 || hi2, e3 = lo3 || hi3;
  if (e1 && (hf >> (hi1 ? 1 : 0) & 1u)) return hi1 ? 1 : 0;
  if (e2 && (hf >> (hi2 ? 3 : 2) & 1u)) return hi2 ? 3 : 2;
  if (e3 && (hf >> (hi3 ? 5 : 4) & 1u)) return hi3 ? 5 : 4;
  if (e2 && e3) {  // edge along x: u = y, v = z
    const int e = 2 * (hi3 ? 1 : 0) + (hi2 ? 1 : 0);
    if (he >> e & 1u) return 6 + e;
  }
  if (e1 && e3) {  // edge along y: u = x, v = z
    const int e = 4 + 2 * (hi3 ? 1 : 0) + (hi1 ? 1 : 0);
    if (he >> e & 1u) return 6 + e;
  }
  if (e1 && e2) {  // edge along z: u = x, v = y
    const int e = 8 + 2 * (hi2 ? 1 : 0) + (hi1 ? 1 : 0);
    if (he >> e & 1u) return 6 + e;
  }
  return -1;
}

// Value at local node (a1, a2, a3) of its owner's interpolation from the coarse values in HB (per cell:
// 6 faces x n^2, u fastest, then 12 edges x n).
template <int N, typename Real>
__device__ __forceinline__ Real hang_value(const Real* P, uint32_t hf, uint32_t he, int own, int a1, int a2, int a3,
                                           const Real* HB) {
  constexpr int N2 = N * N;
  const int a[3] = {a1, a2, a3};
  if (own < 6) {
    const int d = own >> 1, u = d == 0 ? 1 : 0, v = d == 2 ? 1 : 2;
    const int cu = (hf >> (6 + 2 * own)) & 1, cv = (hf >> (7 + 2 * own)) & 1;
    const Real* Pu = P + cu * N2 + a[u] * N;
    const Real* Pv = P + cv * N2 + a[v] * N;
    const Real* F = HB + own * N2;
    Real s = Real(0);
#pragma unroll
    for (int mv = 0; mv < N; ++mv) {
      Real t = Real(0);
#pragma unroll
      for (int mu = 0; mu < N; ++mu) t += Pu[mu] * F[mu + N * mv];
      s += Pv[mv] * t;
    }
    return s;
  }
  const int e = own - 6, d = e >> 2;
  const int cd = (he >> (12 + e)) & 1;
  const Real* Pd = P + cd * N2 + a[d] * N;
  const Real* E = HB + 6 * N2 + e * N;
  Real s = Real(0);
#pragma unroll
  for (int md = 0; md < N; ++md) s += Pd[md] * E[md];
  return s;
}

template <int N>
struct VmultShape {
  static constexpr int NP = (N % 2) ? N : N + 1;  // padded row length (odd)
  static constexpr int N2 = N * N;
  static constexpr int N3 = N * N * N;
  static constexpr int THREADS = 256;
  static constexpr int CB = THREADS / N2;         // cells per CTA step
  static constexpr int CELL = N * N * NP;         // shared elements per cube
};

// The 1D matrices are compile-time constants (generated at build time from the library's
// own rules, basis_tables.h), so every contraction is a chain of FMAs with immediate
// operands: S[q*N + j] = l_j(xi_q) (GLL basis at Gauss points), D[q*N + p] = L_p'(xi_q)
// (collocation derivative on the Gauss points), Sd[q*N + j] = l_j'(xi_q) (derivative of the GLL
// basis at the Gauss points, Sd = D S).
enum { MAT_S = 0, MAT_D = 1, MAT_SD = 2 };

template <int N, int MAT>
__device__ __forceinline__ constexpr double basis_entry(int i) {
  return MAT == MAT_S ? BasisConst<N>::S(i) : MAT == MAT_D ? BasisConst<N>::D(i) : BasisConst<N>::Sd(i);
}

// out = M in
template <int N, typename Real, int MAT>
__device__ __forceinline__ void contract(const Real (&in)[N], Real (&out)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    Real s = Real(basis_entry<N, MAT>(i * N)) * in[0];
#pragma unroll
    for (int j = 1; j < N; ++j) s += Real(basis_entry<N, MAT>(i * N + j)) * in[j];
    out[i] = s;
  }
}

// out = M^T in
template <int N, typename Real, int MAT>
__device__ __forceinline__ void contract_t(const Real (&in)[N], Real (&out)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    Real s = Real(basis_entry<N, MAT>(i)) * in[0];
#pragma unroll
    for (int j = 1; j < N; ++j) s += Real(basis_entry<N, MAT>(j * N + i)) * in[j];
    out[i] = s;
  }
}

// x-line gather of cell `cell` at (i2, i3) through the cell's index table, with constraint
// resolution (hanging: weighted masters; Dirichlet: no masters, value 0).
template <int N, typename Real>
__device__ __forceinline__ void gather_xline(const VmultArgs<N, Real>& a, const Real* __restrict__ src,
                                             int64_t cell, int i2, int i3, Real (&v)[N]) {
  const int32_t* cd = a.cell_dofs + cell * (N * N * N) + (i3 * N + i2) * N;
#pragma unroll
  for (int i1 = 0; i1 < N; ++i1) {
    const int32_t e = __ldg(cd + i1);
    if (e >= 0) {
      v[i1] = __ldg(src + e);
    } else {
      const int32_t row = -e - 1;
      Real s = Real(0);
      for (int64_t p = a.cptr[row]; p < a.cptr[row + 1]; ++p) s += a.cweight[p] * __ldg(src + a.cmaster[p]);
      v[i1] = s;
    }
  }
}

// x-line scatter: the transpose of the gather (atomics into the free DoFs).
template <int N, typename Real>
__device__ __forceinline__ void scatter_xline(const VmultArgs<N, Real>& a, Real* __restrict__ dst, int64_t cell,
                                              int i2, int i3, const Real (&v)[N]) {
  const int32_t* cd = a.cell_dofs + cell * (N * N * N) + (i3 * N + i2) * N;
#pragma unroll
  for (int i1 = 0; i1 < N; ++i1) {
    const int32_t e = __ldg(cd + i1);
    if (e >= 0) {
      atomicAdd(dst + e, v[i1]);
    } else {
      const int32_t row = -e - 1;
      for (int64_t p = a.cptr[row]; p < a.cptr[row + 1]; ++p) atomicAdd(dst + a.cmaster[p], a.cweight[p] * v[i1]);
    }
  }
}

// HANG: the mesh has hanging nodes and its constraints are applied in tensor-product form (a separate
// instantiation, so meshes without them keep the registers and the occupancy of the plain kernel;
// bounded to 80 registers for three CTAs per SM: k = 3 / 4 / 6 16.2 / 17.1 / 17.7 -> 18.1 / 19.7 / 22.0
// GDoF/s on octrees refined twice)
template <int N, typename Real, bool HANG>
__global__ void __launch_bounds__(256, HANG ? 3 : 1) vmult_kernel(const __grid_constant__ VmultArgs<N, Real> a,
                                                    const Real* __restrict__ src, Real* __restrict__ dst) {
  using Sh = VmultShape<N>;
  constexpr int NP = Sh::NP, N2 = Sh::N2, N3 = Sh::N3, CB = Sh::CB, CELL = Sh::CELL;
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* buf0 = reinterpret_cast<Real*>(smem_raw);
  Real* buf1 = buf0 + CB * CELL;
  Real* buf2 = buf1 + CB * CELL;
  Real* hbuf = buf2 + CB * CELL;  // coarse values of hanging faces and edges: CB x (6 n^2 + 12 n)
  constexpr int HB_CELL = 6 * N2 + 12 * N;

  const int t = threadIdx.x;
  const int cl = t / N2;
  const int r = t - cl * N2;
  const int ra = r % N, rb = r / N;  // fast and slow line coordinates
  const bool line_ok = t < CB * N2;
  Real* B0 = buf0 + cl * CELL;
  Real* B1 = buf1 + cl * CELL;
  Real* B2 = buf2 + cl * CELL;

  const int64_t n_items = a.cell_list ? a.n_list : a.n_cells;
  const int64_t nbatch = (n_items + CB - 1) / CB;
  for (int64_t b = blockIdx.x; b < nbatch; b += gridDim.x) {
    const int64_t item = b * CB + cl;
    const bool act = line_ok && item < n_items;
    const int64_t cell = act && a.cell_list ? (int64_t)__ldg(a.cell_list + item) : item;
    Real g3[N], t3[N];
    // hanging faces / edges of this thread's cell (tensor-product constraints, when given)
    const uint32_t hf = (HANG && act) ? __ldg(a.hface + cell) : 0u;
    const uint32_t he = (HANG && act) ? __ldg(a.hedge + cell) : 0u;
    const bool hang = (hf | he) != 0u;
    const bool any_hang = HANG && __syncthreads_or(hang);
    Real* HB = hbuf + (line_ok ? cl : 0) * HB_CELL;

    // 1) gather + S along x: x-line (i2 = ra, i3 = rb)
    if (!any_hang) {
      if (act) {
        Real v[N], o[N];
        gather_xline<N, Real>(a, src, cell, ra, rb, v);
        contract<N, Real, MAT_S>(v, o);
        Real* p = B0 + (rb * N + ra) * NP;
#pragma unroll
        for (int q = 0; q < N; ++q) p[q] = o[q];
      }
    } else {
      // free DoFs directly; constrained nodes owned by a hanging face or edge are interpolated from the
      // coarse values once every thread of the cell has staged them; other constrained nodes as before
      Real v[N];
      int own[N];
      if (act) {
        const int32_t* cd = a.cell_dofs + cell * N3 + (rb * N + ra) * N;
#pragma unroll
        for (int i1 = 0; i1 < N; ++i1) {
          const int32_t e = __ldg(cd + i1);
          own[i1] = (e < 0 && hang) ? hang_owner(hf, he, i1, ra, rb, N - 1) : -1;
          if (e >= 0) {
            v[i1] = __ldg(src + e);
          } else if (own[i1] >= 0) {
            v[i1] = Real(0);
          } else {
            const int32_t row = -e - 1;
            Real s = Real(0);
            for (int64_t p = a.cptr[row]; p < a.cptr[row + 1]; ++p) s += a.cweight[p] * __ldg(src + a.cmaster[p]);
            v[i1] = s;
          }
        }
      }
      if (act && hang) {
        const int64_t h0 = __ldg(a.hoff + cell);
        int slot = 0;
        for (int f = 0; f < 6; ++f) {
          if (!(hf >> f & 1u)) continue;
          const int32_t hd = __ldg(a.hdofs + h0 + slot + r);
          HB[f * N2 + r] = hd >= 0 ? __ldg(src + hd) : Real(0);
          slot += N2;
        }
        for (int e = 0; e < 12; ++e) {
          if (!(he >> e & 1u)) continue;
          if (r < N) {
            const int32_t hd = __ldg(a.hdofs + h0 + slot + r);
            HB[6 * N2 + e * N + r] = hd >= 0 ? __ldg(src + hd) : Real(0);
          }
          slot += N;
        }
      }
      __syncthreads();
      if (act) {
        if (hang) {
#pragma unroll
          for (int i1 = 0; i1 < N; ++i1)
            if (own[i1] >= 0) v[i1] = hang_value<N, Real>(a.P, hf, he, own[i1], i1, ra, rb, HB);
        }
        Real o[N];
        contract<N, Real, MAT_S>(v, o);
        Real* p = B0 + (rb * N + ra) * NP;
#pragma unroll
        for (int q = 0; q < N; ++q) p[q] = o[q];
      }
    }
    __syncthreads();
    // 2) S along y: y-line (q1 = ra, i3 = rb)
    if (act) {
      Real v[N], o[N];
      Real* p = B0 + rb * N * NP + ra;
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = p[j * NP];
      contract<N, Real, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) p[j * NP] = o[j];
    }
    __syncthreads();
    // 3) S along z, then D along z in registers: z-line (q1 = ra, q2 = rb)
    if (act) {
      Real v[N], o[N];
      Real* p = B0 + rb * NP + ra;
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = p[j * N * NP];
      contract<N, Real, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) p[j * N * NP] = o[j];
      contract<N, Real, MAT_D>(o, g3);
    }
    __syncthreads();
    // 4) D along x -> B1 (x-line q2 = ra, q3 = rb); D along y -> B2 (y-line q1 = ra, q3 = rb)
    if (act) {
      Real v[N], o[N];
      const Real* p = B0 + (rb * N + ra) * NP;
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = p[j];
      contract<N, Real, MAT_D>(v, o);
      Real* w = B1 + (rb * N + ra) * NP;
#pragma unroll
      for (int j = 0; j < N; ++j) w[j] = o[j];
      const Real* py = B0 + rb * N * NP + ra;
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = py[j * NP];
      contract<N, Real, MAT_D>(v, o);
      Real* wy = B2 + rb * N * NP + ra;
#pragma unroll
      for (int j = 0; j < N; ++j) wy[j * NP] = o[j];
    }
    __syncthreads();
    // 5) quadrature-point metric on the z-line (q1 = ra, q2 = rb); D_z^T in registers
    if (act) {
      const Real* G = a.metric + cell * (6 * N3) + rb * N + ra;
      Real h3[N];
#pragma unroll
      for (int q3 = 0; q3 < N; ++q3) {
        const int off = q3 * N2;
        const Real G00 = __ldg(G + off), G01 = __ldg(G + N3 + off), G02 = __ldg(G + 2 * N3 + off);
        const Real G11 = __ldg(G + 3 * N3 + off), G12 = __ldg(G + 4 * N3 + off), G22 = __ldg(G + 5 * N3 + off);
        const int sidx = (q3 * N + rb) * NP + ra;
        const Real u1 = B1[sidx], u2 = B2[sidx], u3 = g3[q3];
        B1[sidx] = G00 * u1 + G01 * u2 + G02 * u3;
        B2[sidx] = G01 * u1 + G11 * u2 + G12 * u3;
        h3[q3] = G02 * u1 + G12 * u2 + G22 * u3;
      }
      contract_t<N, Real, MAT_D>(h3, t3);
    }
    __syncthreads();
    // 6) D_x^T on B1 in place (x-line q2 = ra, q3 = rb)
    if (act) {
      Real v[N], o[N];
      Real* p = B1 + (rb * N + ra) * NP;
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = p[j];
      contract_t<N, Real, MAT_D>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) p[j] = o[j];
    }
    __syncthreads();
    // 7) D_y^T on B2, added into B1 (y-line q1 = ra, q3 = rb)
    if (act) {
      Real v[N], o[N];
      Real* p2 = B2 + rb * N * NP + ra;
      Real* p1 = B1 + rb * N * NP + ra;
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = p2[j * NP];
      contract_t<N, Real, MAT_D>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) p1[j * NP] += o[j];
    }
    __syncthreads();
    // 8) add D_z^T h3, then S_z^T (z-line q1 = ra, q2 = rb)
    if (act) {
      Real v[N], o[N];
      Real* p = B1 + rb * NP + ra;
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = p[j * N * NP] + t3[j];
      contract_t<N, Real, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) p[j * N * NP] = o[j];
    }
    __syncthreads();
    // 9) S_y^T (y-line i1 = ra, i3 = rb)
    if (act) {
      Real v[N], o[N];
      Real* p = B1 + rb * N * NP + ra;
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = p[j * NP];
      contract_t<N, Real, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) p[j * NP] = o[j];
    }
    __syncthreads();
    // 10) S_x^T and scatter (x-line i2 = ra, i3 = rb)
    if (!any_hang) {
      if (act) {
        Real v[N], o[N];
        const Real* p = B1 + (rb * N + ra) * NP;
#pragma unroll
        for (int j = 0; j < N; ++j) v[j] = p[j];
        contract_t<N, Real, MAT_S>(v, o);
        scatter_xline<N, Real>(a, dst, cell, ra, rb, o);
      }
    } else {
      // nodes owned by a hanging face or edge go to the coarse DoFs through the transposed interpolation
      // (staged in B0, which phase 4 last read); the other nodes are scattered as before
      if (act) {
        Real v[N], o[N];
        const Real* p = B1 + (rb * N + ra) * NP;
#pragma unroll
        for (int j = 0; j < N; ++j) v[j] = p[j];
        contract_t<N, Real, MAT_S>(v, o);
        const int32_t* cd = a.cell_dofs + cell * N3 + (rb * N + ra) * N;
        Real* w = B0 + (rb * N + ra) * NP;
#pragma unroll
        for (int i1 = 0; i1 < N; ++i1) {
          const int32_t e = __ldg(cd + i1);
          const int own = (e < 0 && hang) ? hang_owner(hf, he, i1, ra, rb, N - 1) : -1;
          w[i1] = own >= 0 ? o[i1] : Real(0);
          if (own >= 0) continue;
          if (e >= 0) {
            atomicAdd(dst + e, o[i1]);
          } else {
            const int32_t row = -e - 1;
            for (int64_t q = a.cptr[row]; q < a.cptr[row + 1]; ++q) atomicAdd(dst + a.cmaster[q], a.cweight[q] * o[i1]);
          }
        }
      }
      __syncthreads();
      if (act && hang) {
        constexpr int K = N - 1;
        const int64_t h0 = __ldg(a.hoff + cell);
        int slot = 0;
        for (int f = 0; f < 6; ++f) {
          if (!(hf >> f & 1u)) continue;
          // coarse face node (mu, mv) = (r % N, r / N): sum over the fine face nodes this face owns
          const int d = f >> 1, u = d == 0 ? 1 : 0, v = d == 2 ? 1 : 2;
          const int cu = (hf >> (6 + 2 * f)) & 1, cv = (hf >> (7 + 2 * f)) & 1;
          const int mu = r % N, mv = r / N;
          const Real* Pu = a.P + cu * N2 + mu;
          const Real* Pv = a.P + cv * N2 + mv;
          const int step[3] = {1, NP, N * NP};
          const int base = (f & 1) * K * step[d];
          Real s = Real(0);
          for (int bv = 0; bv < N; ++bv) {
            // face f owns node (bu, bv) unless a hanging face of lower index also contains it
            const int sv = bv == 0 ? 0 : (bv == K ? 1 : -1);
            if (sv >= 0 && 2 * v + sv < f && (hf >> (2 * v + sv) & 1u)) continue;
            Real t = Real(0);
            for (int bu = 0; bu < N; ++bu) {
              const int su = bu == 0 ? 0 : (bu == K ? 1 : -1);
              if (su >= 0 && 2 * u + su < f && (hf >> (2 * u + su) & 1u)) continue;
              t += Pu[bu * N] * B0[base + bu * step[u] + bv * step[v]];
            }
            s += Pv[bv * N] * t;
          }
          const int32_t hd = __ldg(a.hdofs + h0 + slot + r);
          if (hd >= 0) atomicAdd(dst + hd, s);
          slot += N2;
        }
        for (int e = 0; e < 12; ++e) {
          if (!(he >> e & 1u)) continue;
          if (r < N) {
            const int d = e >> 2, u = d == 0 ? 1 : 0, v = d == 2 ? 1 : 2;
            const int cdh = (he >> (12 + e)) & 1;
            Real s = Real(0);
            for (int bd = 0; bd < N; ++bd) {
              int aa[3];
              aa[d] = bd;
              aa[u] = (e & 1) * K;
              aa[v] = ((e >> 1) & 1) * K;
              if (hang_owner(hf, he, aa[0], aa[1], aa[2], K) != 6 + e) continue;
              s += a.P[cdh * N2 + bd * N + r] * B0[(aa[2] * N + aa[1]) * NP + aa[0]];
            }
            const int32_t hd = __ldg(a.hdofs + h0 + slot + r);
            if (hd >= 0) atomicAdd(dst + hd, s);
          }
          slot += N;
        }
      }
    }
    __syncthreads();
  }
}

// dst = src on constrained rows, 0 elsewhere (identity rows of the condensed operator).
template <int N, typename Real>
__global__ void vmult_prologue(const __grid_constant__ VmultArgs<N, Real> a, const Real* __restrict__ src,
                               Real* __restrict__ dst) {
  if (a.skip && *a.skip) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t i0 = 0;
  // four DoFs per step where src and dst allow 4-element vector stores (the mask is the library's own,
  // 256-byte aligned): one 4-byte mask load, src read only on constrained DoFs
  if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & (4 * sizeof(Real) - 1)) == 0) {
    const int64_t n4 = a.n_dofs >> 2;
    for (int64_t i = tid; i < n4; i += stride) {
      const uchar4 m = reinterpret_cast<const uchar4*>(a.cmask)[i];
      const Real* s = src + 4 * i;
      const Real v0 = m.x ? s[0] : Real(0), v1 = m.y ? s[1] : Real(0);
      const Real v2 = m.z ? s[2] : Real(0), v3 = m.w ? s[3] : Real(0);
      if constexpr (sizeof(Real) == 4) {
        reinterpret_cast<float4*>(dst)[i] = make_float4(v0, v1, v2, v3);
      } else {
        reinterpret_cast<double2*>(dst)[2 * i] = make_double2(v0, v1);
        reinterpret_cast<double2*>(dst)[2 * i + 1] = make_double2(v2, v3);
      }
    }
    i0 = 4 * n4;
  }
  for (int64_t i = i0 + tid; i < a.n_dofs; i += stride) dst[i] = a.cmask[i] != 0 ? src[i] : Real(0);
}

}  // namespace mfx
