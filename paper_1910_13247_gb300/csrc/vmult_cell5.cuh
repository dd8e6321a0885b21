// Per-cell vmult in five synchronised phases on meshes with index tables (octrees, hanging nodes): the
// operator of Sec. 3.6 with the tensor-product evaluation of Sec. 3.1 and the constraints of Sec. 3.3
// resolved in the gather and its transpose in the scatter (hanging nodes per node through their
// masters, or, with HANG, in tensor-product form on the cells listed as having hanging faces or edges:
// the coarse face and edge values are interpolated to the fine nodes, Fig. 2).
//
// The reference gradient at the Gauss points is taken with the derivative of the nodal basis at the
// Gauss points, Sd[q][j] = l_j'(xi_q), next to its values S[q][j] = l_j(xi_q), so every line of a
// direction is read from shared memory once and both of its contractions come from the same registers
// (the structure of the five-phase row kernel, vmult_brick_f5.cuh, one cell per line instead of a pair):
//   1) x-lines (gather through the index table):  A = S_x u,  C = Sd_x u
//   2) y-lines:  A <- S_y A,  B = Sd_y A,  C <- S_y C
//   3) z-lines:  grad = (S_z C, S_z B, Sd_z A) at the Gauss points, h = G_q grad (G_q the merged metric,
//      read once, coalesced), then C <- S_z^T h_1, B <- S_z^T h_2, A <- Sd_z^T h_3, all in registers
//   4) y-lines:  A <- S_y^T A + Sd_y^T B,  C <- S_y^T C
//   5) x-lines:  out = S_x^T A + Sd_x^T C, added into dst with atomics through the index table
// Sixteen 1D contractions per line in five phases, against fifteen in ten phases (vmult_kernel): half
// the barriers and fewer shared-memory accesses per line.  Without hanging cells a thread's phase-5
// reads and the next batch's phase-1 writes touch only its own x-line, so no barrier closes a batch.
// dst must hold src on the constrained rows and 0 elsewhere before the launch (vmult_prologue).
#pragma once

#include "vmult.cuh"

namespace mfx {

// sum_j M[q][j] in[j]
template <int N, typename Real, int MAT>
__device__ __forceinline__ Real row1(const Real (&in)[N], int q) {
  Real s = Real(basis_entry<N, MAT>(q * N)) * in[0];
#pragma unroll
  for (int j = 1; j < N; ++j) s += Real(basis_entry<N, MAT>(q * N + j)) * in[j];
  return s;
}

// acc[i] (+)= M[q][i] h   (column q of M^T)
template <int N, typename Real, int MAT>
__device__ __forceinline__ void axpy_col1(Real (&acc)[N], Real h, int q, bool first) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const Real m = Real(basis_entry<N, MAT>(q * N + i));
    acc[i] = first ? m * h : acc[i] + m * h;
  }
}

// out = M1^T a + M2^T b
template <int N, typename Real, int M1, int M2>
__device__ __forceinline__ void contract_tt1(const Real (&x)[N], const Real (&y)[N], Real (&out)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    Real s = Real(basis_entry<N, M1>(i)) * x[0];
#pragma unroll
    for (int j = 1; j < N; ++j) s += Real(basis_entry<N, M1>(j * N + i)) * x[j];
#pragma unroll
    for (int j = 0; j < N; ++j) s += Real(basis_entry<N, M2>(j * N + i)) * y[j];
    out[i] = s;
  }
}

// Scratch of the tensor-product interpolation of hanging values (per cell 6 n^2 + 12 n values): the B and
// C cubes of the cell where they are large enough, else a region of its own after the coarse values
template <int N>
struct Cell5Scratch {
  static constexpr bool OWN = 2 * VmultShape<N>::CELL < 6 * N * N + 12 * N;
};

// HANG: hanging constraints in tensor-product form (bounded to 80 registers for three CTAs per SM, as
// the ten-phase kernel)
template <int N, typename Real, bool HANG, bool BOX = false>
__global__ void __launch_bounds__(256, HANG ? 3 : (sizeof(Real) == 4 ? 4 : 1)) vmult5_kernel(const __grid_constant__ VmultArgs<N, Real> a,
                                                                    const Real* __restrict__ src,
                                                                    Real* __restrict__ dst) {
  using Sh = VmultShape<N>;
  constexpr int NP = Sh::NP, N2 = Sh::N2, N3 = Sh::N3, CB = Sh::CB, CELL = Sh::CELL;
  constexpr int HB_CELL = 6 * N2 + 12 * N;  // coarse values of hanging faces and edges per cell
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int t = threadIdx.x;
  const int cl = t / N2;
  const int r = t - cl * N2;
  const int ra = r % N, rb = r / N;  // fast and slow line coordinates
  const bool line_ok = t < CB * N2;
  // three cubes per cell, [i3][i2][i1] with rows padded to NP (odd): every line access is conflict-free
  Real* A = reinterpret_cast<Real*>(smem_raw) + (line_ok ? cl : 0) * CELL;
  Real* B = A + CB * CELL;
  Real* C = B + CB * CELL;
  Real* const B0 = reinterpret_cast<Real*>(smem_raw) + CB * CELL;  // the B and C cubes of all cells
  Real* HB = reinterpret_cast<Real*>(smem_raw) + 3 * CB * CELL + (line_ok ? cl : 0) * HB_CELL;

  const int xl = (rb * N + ra) * NP;  // x-line (i2 = ra, i3 = rb)
  const int yl = rb * N * NP + ra;    // y-line (x = ra, z = rb), stride NP
  const int zl = rb * NP + ra;        // z-line (x = ra, y = rb), stride N NP

  const int64_t n_items = a.cell_list ? a.n_list : a.n_cells;
  const int64_t nbatch = (n_items + CB - 1) / CB;
  for (int64_t b = blockIdx.x; b < nbatch; b += gridDim.x) {
    const int64_t item = b * CB + cl;
    const bool act = line_ok && item < n_items;
    const int64_t cell = act && a.cell_list ? (int64_t)__ldg(a.cell_list + item) : item;
    // hanging faces / edges of this thread's cell (tensor-product constraints)
    const uint32_t hf = (HANG && act) ? __ldg(a.hface + cell) : 0u;
    const uint32_t he = (HANG && act) ? __ldg(a.hedge + cell) : 0u;
    const bool hang = (hf | he) != 0u;
    const bool any_hang = HANG && __syncthreads_or(hang);
    // 1) x-lines: gather, A = S_x u, C = Sd_x u
    Real v[N];
    if (!HANG || !any_hang) {
      if (act) gather_xline<N, Real>(a, src, cell, ra, rb, v);
    } else {
      // free DoFs directly; constrained nodes owned by a hanging face or edge are interpolated from the
      // coarse values once every thread of the cell has staged them; other constrained nodes through
      // their masters
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
      // the coarse values interpolated to the fine face and edge nodes in tensor-product form, N^3 instead
      // of N^4 multiply-adds per face: along u into the scratch TS (B and C, free until the contractions
      // of this phase), then along v back into HB; an edge's 1D interpolation goes through TS unchanged
      Real* TS = Cell5Scratch<N>::OWN ? HB + CB * HB_CELL : B0 + (line_ok ? cl : 0) * 2 * CELL;
      if (act && hang) {
        const int au = r % N, mw = r / N;
        for (int f = 0; f < 6; ++f) {
          if (!(hf >> f & 1u)) continue;
          const Real* Pu = a.P + ((hf >> (6 + 2 * f)) & 1) * N2 + au * N;
          const Real* F = HB + f * N2 + N * mw;
          Real t = Real(0);
#pragma unroll
          for (int mu = 0; mu < N; ++mu) t += Pu[mu] * F[mu];
          TS[f * N2 + r] = t;
        }
        if (r < N)
          for (int e = 0; e < 12; ++e) {
            if (!(he >> e & 1u)) continue;
            const Real* Pd = a.P + ((he >> (12 + e)) & 1) * N2 + r * N;
            const Real* E = HB + 6 * N2 + e * N;
            Real t = Real(0);
#pragma unroll
            for (int md = 0; md < N; ++md) t += Pd[md] * E[md];
            TS[6 * N2 + e * N + r] = t;
          }
      }
      __syncthreads();
      if (act && hang) {
        const int au = r % N, av = r / N;
        for (int f = 0; f < 6; ++f) {
          if (!(hf >> f & 1u)) continue;
          const Real* Pv = a.P + ((hf >> (7 + 2 * f)) & 1) * N2 + av * N;
          const Real* Tf = TS + f * N2 + au;
          Real t = Real(0);
#pragma unroll
          for (int mv = 0; mv < N; ++mv) t += Pv[mv] * Tf[N * mv];
          HB[f * N2 + r] = t;
        }
        if (r < N)
          for (int e = 0; e < 12; ++e)
            if (he >> e & 1u) HB[6 * N2 + e * N + r] = TS[6 * N2 + e * N + r];
      }
      __syncthreads();
      if (act && hang) {
#pragma unroll
        for (int i1 = 0; i1 < N; ++i1) {
          const int o = own[i1];
          if (o < 0) continue;
          const int ac[3] = {i1, ra, rb};
          if (o < 6) {
            const int d = o >> 1, u = d == 0 ? 1 : 0, w = d == 2 ? 1 : 2;
            v[i1] = HB[o * N2 + ac[u] + N * ac[w]];
          } else {
            v[i1] = HB[6 * N2 + (o - 6) * N + ac[(o - 6) >> 2]];
          }
        }
      }
    }
    if (act) {
      Real o[N];
      contract<N, Real, MAT_S>(v, o);
#pragma unroll
      for (int q = 0; q < N; ++q) A[xl + q] = o[q];
      contract<N, Real, MAT_SD>(v, o);
#pragma unroll
      for (int q = 0; q < N; ++q) C[xl + q] = o[q];
    }
    __syncthreads();
    // 2) y-lines: A <- S_y A, B = Sd_y A, C <- S_y C
    if (act) {
      Real v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[yl + j * NP];
      contract<N, Real, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[yl + j * NP] = o[j];
      contract<N, Real, MAT_SD>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) B[yl + j * NP] = o[j];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = C[yl + j * NP];
      contract<N, Real, MAT_S>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) C[yl + j * NP] = o[j];
    }
    __syncthreads();
    // 3) z-lines: gradient at the Gauss points, metric, transposed z-contractions, in registers
    if (act) {
      Real va[N], vb[N], vc[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        va[j] = A[zl + j * N * NP];
        vb[j] = B[zl + j * N * NP];
        vc[j] = C[zl + j * N * NP];
      }
      Real oa[N], ob[N], oc[N];
      if constexpr (BOX) {
        // box cell: metric w_q diag(D), one D per cell, the weights of the line's point (ra, rb) times
        // the z-weight of each point
        const float* Db = a.box + cell * 3;
        const Real wab = a.wq[ra] * a.wq[rb];
        const Real D0 = wab * __ldg(Db), D1 = wab * __ldg(Db + 1), D2 = wab * __ldg(Db + 2);
#pragma unroll
        for (int q3 = 0; q3 < N; ++q3) {
          const Real u1 = row1<N, Real, MAT_S>(vc, q3);   // d/dx
          const Real u2 = row1<N, Real, MAT_S>(vb, q3);   // d/dy
          const Real u3 = row1<N, Real, MAT_SD>(va, q3);  // d/dz
          const Real wz = a.wq[q3];
          axpy_col1<N, Real, MAT_S>(oc, (D0 * wz) * u1, q3, q3 == 0);
          axpy_col1<N, Real, MAT_S>(ob, (D1 * wz) * u2, q3, q3 == 0);
          axpy_col1<N, Real, MAT_SD>(oa, (D2 * wz) * u3, q3, q3 == 0);
        }
      } else {
        const Real* G = a.metric + cell * (6 * N3) + rb * N + ra;
#pragma unroll
        for (int q3 = 0; q3 < N; ++q3) {
          const Real u1 = row1<N, Real, MAT_S>(vc, q3);   // d/dx
          const Real u2 = row1<N, Real, MAT_S>(vb, q3);   // d/dy
          const Real u3 = row1<N, Real, MAT_SD>(va, q3);  // d/dz
          const int off = q3 * N2;
          const Real G00 = __ldg(G + off), G01 = __ldg(G + N3 + off), G02 = __ldg(G + 2 * N3 + off);
          const Real G11 = __ldg(G + 3 * N3 + off), G12 = __ldg(G + 4 * N3 + off), G22 = __ldg(G + 5 * N3 + off);
          const Real h1 = G00 * u1 + G01 * u2 + G02 * u3;
          const Real h2 = G01 * u1 + G11 * u2 + G12 * u3;
          const Real h3 = G02 * u1 + G12 * u2 + G22 * u3;
          axpy_col1<N, Real, MAT_S>(oc, h1, q3, q3 == 0);
          axpy_col1<N, Real, MAT_S>(ob, h2, q3, q3 == 0);
          axpy_col1<N, Real, MAT_SD>(oa, h3, q3, q3 == 0);
        }
      }
#pragma unroll
      for (int j = 0; j < N; ++j) {
        A[zl + j * N * NP] = oa[j];
        B[zl + j * N * NP] = ob[j];
        C[zl + j * N * NP] = oc[j];
      }
    }
    __syncthreads();
    // 4) y-lines: A <- S_y^T A + Sd_y^T B, C <- S_y^T C
    if (act) {
      Real va[N], vb[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        va[j] = A[yl + j * NP];
        vb[j] = B[yl + j * NP];
      }
      contract_tt1<N, Real, MAT_S, MAT_SD>(va, vb, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[yl + j * NP] = o[j];
#pragma unroll
      for (int j = 0; j < N; ++j) va[j] = C[yl + j * NP];
      contract_t<N, Real, MAT_S>(va, o);
#pragma unroll
      for (int j = 0; j < N; ++j) C[yl + j * NP] = o[j];
    }
    __syncthreads();
    // 5) x-lines: out = S_x^T A + Sd_x^T C, scattered
    if (act) {
      Real va[N], vc[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        va[j] = A[xl + j];
        vc[j] = C[xl + j];
      }
      contract_tt1<N, Real, MAT_S, MAT_SD>(va, vc, o);
      if (!HANG || !any_hang) {
        scatter_xline<N, Real>(a, dst, cell, ra, rb, o);
      } else {
        // nodes owned by a hanging face or edge go to the coarse DoFs through the transposed
        // interpolation (staged in B, which phase 4 last read); the other nodes are scattered as before
        const int32_t* cd = a.cell_dofs + cell * N3 + (rb * N + ra) * N;
#pragma unroll
        for (int i1 = 0; i1 < N; ++i1) {
          const int32_t e = __ldg(cd + i1);
          const int own = (e < 0 && hang) ? hang_owner(hf, he, i1, ra, rb, N - 1) : -1;
          B[xl + i1] = own >= 0 ? o[i1] : Real(0);
          if (own >= 0) continue;
          if (e >= 0) {
            atomicAdd(dst + e, o[i1]);
          } else {
            const int32_t row = -e - 1;
            for (int64_t q = a.cptr[row]; q < a.cptr[row + 1]; ++q) atomicAdd(dst + a.cmaster[q], a.cweight[q] * o[i1]);
          }
        }
      }
    }
    if (HANG && any_hang) {
      __syncthreads();
      constexpr int K = N - 1;
      const int step[3] = {1, NP, N * NP};
      // the transposed interpolation onto the coarse face DoFs in tensor-product form: along u into HB
      // (free since the gather), then along v; a fine node on a hanging face of lower index belongs to
      // that face and adds nothing here
      if (act && hang) {
        const int mu = r % N, bv = r / N;
        const int sv = bv == 0 ? 0 : (bv == K ? 1 : -1);
        for (int f = 0; f < 6; ++f) {
          if (!(hf >> f & 1u)) continue;
          const int d = f >> 1, u = d == 0 ? 1 : 0, w = d == 2 ? 1 : 2;
          Real t = Real(0);
          if (!(sv >= 0 && 2 * w + sv < f && (hf >> (2 * w + sv) & 1u))) {
            const Real* Pu = a.P + ((hf >> (6 + 2 * f)) & 1) * N2 + mu;
            const int base = (f & 1) * K * step[d] + bv * step[w];
            for (int bu = 0; bu < N; ++bu) {
              const int su = bu == 0 ? 0 : (bu == K ? 1 : -1);
              if (su >= 0 && 2 * u + su < f && (hf >> (2 * u + su) & 1u)) continue;
              t += Pu[bu * N] * B[base + bu * step[u]];
            }
          }
          HB[f * N2 + r] = t;
        }
      }
      __syncthreads();
      if (act && hang) {
        const int64_t h0 = __ldg(a.hoff + cell);
        int slot = 0;
        const int mu = r % N, mv = r / N;
        for (int f = 0; f < 6; ++f) {
          if (!(hf >> f & 1u)) continue;
          const Real* Pv = a.P + ((hf >> (7 + 2 * f)) & 1) * N2 + mv;
          const Real* Tf = HB + f * N2 + mu;
          Real s = Real(0);
#pragma unroll
          for (int bv = 0; bv < N; ++bv) s += Pv[bv * N] * Tf[N * bv];
          const int32_t hd = __ldg(a.hdofs + h0 + slot + r);
          if (hd >= 0) atomicAdd(dst + hd, s);
          slot += N2;
        }
        for (int e = 0; e < 12; ++e) {
          if (!(he >> e & 1u)) continue;
          if (r < N) {
            const int d = e >> 2, u = d == 0 ? 1 : 0, w = d == 2 ? 1 : 2;
            const int cdh = (he >> (12 + e)) & 1;
            Real s = Real(0);
            for (int bd = 0; bd < N; ++bd) {
              int aa[3];
              aa[d] = bd;
              aa[u] = (e & 1) * K;
              aa[w] = ((e >> 1) & 1) * K;
              if (hang_owner(hf, he, aa[0], aa[1], aa[2], K) != 6 + e) continue;
              s += a.P[cdh * N2 + bd * N + r] * B[(aa[2] * N + aa[1]) * NP + aa[0]];
            }
            const int32_t hd = __ldg(a.hdofs + h0 + slot + r);
            if (hd >= 0) atomicAdd(dst + hd, s);
          }
          slot += N;
        }
      }
    }
  }
}

}  // namespace mfx
