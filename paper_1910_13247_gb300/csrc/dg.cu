// Symmetric interior penalty DG (SIPG) Laplacian on uniform Cartesian boxes: vmult and diagonal.
//
// The discretisation of the paper's multigrid benchmark (Sec. 6.1): discontinuous Q_k on
// Gauss-Lobatto nodes, DoFs cell-major (cell c, local node i1 + n (i2 + n i3)), a constant
// coefficient a, and
//   a(u, v) = sum_K int_K a grad u . grad v
//           + sum_{interior F} int_F a ( -{d_n u} [v] - [u] {d_n v} + sigma_F [u] [v] )
//           + sum_{Dirichlet F} int_F a ( -(d_n u) v - u (d_n v) + sigma_F u v ),
// n from the lower to the upper cell (outward on the boundary), [w] = w^- - w^+, {w} the mean,
// sigma_F = eta (k+1)^2 / h on interior faces and 2 eta (k+1)^2 / h on Dirichlet faces (h the cell
// size normal to the face), (k+1)-point Gauss quadrature on cells and faces.
//
// Element-centric: a CTA takes CB cells, one thread per line of a cell, and computes each cell's
// output row block on its own, so dst is written once per entry, without atomics:
//   * cell term in Kronecker form, c_x (K1 (x) M1 (x) M1) + c_y (M1 (x) K1 (x) M1) + c_z (M1 (x) M1 (x) K1)
//     with the exact 1D stiffness / mass matrices K1, M1 of the nodal basis (n-point Gauss is exact
//     for them) and c_d = a V / h_d^2: eight 1D sweeps in shared memory;
//   * the six faces in turn: traces (value and normal derivative at the face nodes) of the cell and
//     of the neighbour across the face, interpolated to the face Gauss points, the face integrand, and
//     its transpose back onto the cell's face nodes (value test functions) and onto every node of each
//     normal line (normal-derivative test functions).
#include <algorithm>

#include "mfx_internal.h"

namespace mfx {

int device_sm_count();

struct DgArgs {
  int nx, ny, nz;
  int64_t n_cells;
  double h[3];
  double coef, sig_int[3], sig_bnd[3];
  uint32_t dmask;
  // 1D tables (n <= 9): S[q][i] = l_i(x_q), K1, M1 (n x n), endpoint values / derivatives
  double S[kMaxN * kMaxN], K1[kMaxN * kMaxN], M1[kMaxN * kMaxN], wq[kMaxN];
  double d0[kMaxN], d1[kMaxN];  // l_i'(0), l_i'(1)
  const int32_t* skip;
};

template <typename Real>
__device__ __forceinline__ Real tab(const double* t, int i) {
  return (Real)t[i];
}

// out = M along direction dir (0: i1, 1: i2, 2: i3) of an n^3 cube; thread owns line `line`
template <int N, typename Real>
__device__ __forceinline__ void dg_sweep(const Real* in, Real* out, const double* M, int dir, int line) {
  constexpr int N2 = N * N;
  const int a = line % N, b = line / N;
  const int base = dir == 0 ? N * a + N2 * b : (dir == 1 ? a + N2 * b : a + N * b);
  const int stride = dir == 0 ? 1 : (dir == 1 ? N : N2);
  Real x[N];
#pragma unroll
  for (int i = 0; i < N; ++i) x[i] = in[base + i * stride];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    Real s = Real(0);
#pragma unroll
    for (int j = 0; j < N; ++j) s += tab<Real>(M, i * N + j) * x[j];
    out[base + i * stride] = s;
  }
}

template <int N, typename Real>
__global__ void __launch_bounds__(128) dg_vmult_kernel(const __grid_constant__ DgArgs a, const Real* __restrict__ src,
                                                        Real* __restrict__ dst) {
  constexpr int N2 = N * N, N3 = N2 * N, K = N - 1;
  constexpr int CB = 128 / N2 > 0 ? 128 / N2 : 1;
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sh = reinterpret_cast<Real*>(smem_raw);
  const int cl = threadIdx.x / N2;
  const int r = threadIdx.x - cl * N2;
  const bool lane_ok = cl < CB;
  // per cell: u, y, T1, T2, B1 (n^3 each) and the face buffers (4 traces + 2 integrands, n^2 each)
  Real* u = sh + (size_t)(lane_ok ? cl : 0) * (5 * N3 + 6 * N2);
  Real* y = u + N3;
  Real* T1 = y + N3;
  Real* T2 = T1 + N3;
  Real* B1 = T2 + N3;
  Real* fb = B1 + N3;  // ov, od, nv, nd, fval, fder
  const int64_t nbatch = (a.n_cells + CB - 1) / CB;
  for (int64_t bt = blockIdx.x; bt < nbatch; bt += gridDim.x) {
    const int64_t cell = bt * CB + cl;
    const bool act = lane_ok && cell < a.n_cells;
    const int cx = act ? (int)(cell % a.nx) : 0;
    const int64_t rest = act ? cell / a.nx : 0;
    const int cy = (int)(rest % a.ny), cz = (int)(rest / a.ny);
    const int cidx[3] = {cx, cy, cz};
    const int dims[3] = {a.nx, a.ny, a.nz};
    if (act)
      for (int i = r; i < N3; i += N2) u[i] = src[cell * N3 + i];
    __syncthreads();
    // ---- cell term
    const double vol = a.h[0] * a.h[1] * a.h[2];
    const Real cxf = (Real)(a.coef * vol / (a.h[0] * a.h[0]));
    const Real cyf = (Real)(a.coef * vol / (a.h[1] * a.h[1]));
    const Real czf = (Real)(a.coef * vol / (a.h[2] * a.h[2]));
    if (act) dg_sweep<N, Real>(u, T1, a.K1, 0, r);   // K1_x u
    if (act) dg_sweep<N, Real>(u, B1, a.M1, 0, r);   // M1_x u
    __syncthreads();
    if (act) dg_sweep<N, Real>(T1, T2, a.M1, 1, r);  // M1_y K1_x u
    __syncthreads();
    if (act) dg_sweep<N, Real>(T2, T1, a.M1, 2, r);  // M1_z M1_y K1_x u
    __syncthreads();
    if (act)
      for (int i = r; i < N3; i += N2) y[i] = cxf * T1[i];
    if (act) dg_sweep<N, Real>(B1, T2, a.K1, 1, r);  // K1_y M1_x u
    __syncthreads();
    if (act) dg_sweep<N, Real>(T2, T1, a.M1, 2, r);  // M1_z K1_y M1_x u
    __syncthreads();
    if (act)
      for (int i = r; i < N3; i += N2) y[i] += cyf * T1[i];
    if (act) dg_sweep<N, Real>(B1, T2, a.M1, 1, r);  // M1_y M1_x u
    __syncthreads();
    if (act) dg_sweep<N, Real>(T2, T1, a.K1, 2, r);  // K1_z M1_y M1_x u
    __syncthreads();
    if (act)
      for (int i = r; i < N3; i += N2) y[i] += czf * T1[i];
    __syncthreads();
    // ---- faces
    for (int d = 0; d < 3; ++d) {
      const int e = d == 0 ? 1 : 0, f = d == 2 ? 1 : 2;  // tangential directions (e < f)
      const int st[3] = {1, N, N2};
      const double hd = a.h[d];
      const double area = a.h[e] * a.h[f];
      for (int s = 0; s < 2; ++s) {
        const bool has_nb = s == 1 ? cidx[d] + 1 < dims[d] : cidx[d] > 0;
        const bool dir_face = !has_nb && ((a.dmask >> (2 * d + s)) & 1u);
        // uniform across the CTA's cells only by accident: every thread runs the same sequence of
        // barriers and masks its work
        const int ta = r % N, tb = r / N;  // face node (a, b) = (i_e, i_f)
        const int fbase = ta * st[e] + tb * st[f];
        const double* dl = s == 1 ? a.d1 : a.d0;   // own normal derivative at xi_d = s
        const double* dn = s == 1 ? a.d0 : a.d1;   // neighbour's at xi_d = 1 - s
        if (act && (has_nb || dir_face)) {
          Real od = Real(0);
#pragma unroll
          for (int j = 0; j < N; ++j) od += tab<Real>(dl, j) * u[fbase + j * st[d]];
          fb[0 * N2 + r] = u[fbase + (s * K) * st[d]];
          fb[1 * N2 + r] = od / (Real)hd;
          Real nv = Real(0), nd = Real(0);
          if (has_nb) {
            const int64_t ncell = cell + (s == 1 ? 1 : -1) * (d == 0 ? 1 : (d == 1 ? (int64_t)a.nx : (int64_t)a.nx * a.ny));
            const Real* un = src + ncell * N3;
#pragma unroll
            for (int j = 0; j < N; ++j) nd += tab<Real>(dn, j) * un[fbase + j * st[d]];
            nv = un[fbase + ((1 - s) * K) * st[d]];
          }
          fb[2 * N2 + r] = nv;
          fb[3 * N2 + r] = nd / (Real)hd;
        }
        __syncthreads();
        // integrand at the face Gauss point (qa, qb) = (ta, tb)
        if (act && (has_nb || dir_face)) {
          Real tr[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            Real acc = Real(0);
            for (int j = 0; j < N; ++j) {
              const Real sa = tab<Real>(a.S, ta * N + j);
              for (int l = 0; l < N; ++l) acc += sa * tab<Real>(a.S, tb * N + l) * fb[c * N2 + j + N * l];
            }
            tr[c] = acc;
          }
          const Real w = (Real)(a.coef * area) * tab<Real>(a.wq, ta) * tab<Real>(a.wq, tb);
          Real fval, fder;
          if (has_nb) {
            const Real sig = (Real)a.sig_int[d];
            // own side "-" when the face is the cell's upper face (s = 1)
            const Real Um = s == 1 ? tr[0] : tr[2], Up = s == 1 ? tr[2] : tr[0];
            const Real Dm = s == 1 ? tr[1] : tr[3], Dp = s == 1 ? tr[3] : tr[1];
            const Real J = Um - Up, A = Real(0.5) * (Dm + Dp);
            fval = (s == 1 ? (-A + sig * J) : (A - sig * J)) * w;
            fder = Real(-0.5) * J * w;
          } else {
            const Real sig = (Real)a.sig_bnd[d];
            const Real dnu = s == 1 ? tr[1] : -tr[1];   // outward normal derivative
            fval = (-dnu + sig * tr[0]) * w;
            fder = (s == 1 ? -tr[0] : tr[0]) * w;       // coefficient of d_{+d} v
          }
          fb[4 * N2 + r] = fval;
          fb[5 * N2 + r] = fder;
        }
        __syncthreads();
        // transpose back onto face node (ta, tb) and its normal line
        if (act && (has_nb || dir_face)) {
          Real gv = Real(0), gd = Real(0);
          for (int qa = 0; qa < N; ++qa) {
            const Real sa = tab<Real>(a.S, qa * N + ta);
            for (int qb = 0; qb < N; ++qb) {
              const Real sab = sa * tab<Real>(a.S, qb * N + tb);
              gv += sab * fb[4 * N2 + qa + N * qb];
              gd += sab * fb[5 * N2 + qa + N * qb];
            }
          }
          y[fbase + (s * K) * st[d]] += gv;
          const Real gdh = gd / (Real)hd;
#pragma unroll
          for (int j = 0; j < N; ++j) y[fbase + j * st[d]] += tab<Real>(dl, j) * gdh;
        }
        __syncthreads();
      }
    }
    if (act)
      for (int i = r; i < N3; i += N2) dst[cell * N3 + i] = y[i];
    __syncthreads();
  }
}

// Diagonal: cell term c_x K1_ii M1_jj M1_ll + ... plus, on each face with a term, the self-coupling
// of the face nodes: sum_q w (-+ phi d phi + sigma phi^2) (separable in the 1D mass diagonal).
__global__ void dg_diagonal_kernel(const __grid_constant__ DgArgs a, int n, double* __restrict__ d64,
                                   float* __restrict__ d32) {
  const int n3 = n * n * n, K = n - 1;
  const int64_t total = a.n_cells * n3;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = idx / n3;
    const int i = (int)(idx - cell * n3);
    const int ii[3] = {i % n, (i / n) % n, i / (n * n)};
    const int cidx[3] = {(int)(cell % a.nx), (int)((cell / a.nx) % a.ny), (int)(cell / ((int64_t)a.nx * a.ny))};
    const int dims[3] = {a.nx, a.ny, a.nz};
    const double vol = a.h[0] * a.h[1] * a.h[2];
    double v = 0.0;
    for (int d = 0; d < 3; ++d) {
      double t = a.coef * vol / (a.h[d] * a.h[d]);
      for (int c = 0; c < 3; ++c) t *= c == d ? a.K1[ii[c] * n + ii[c]] : a.M1[ii[c] * n + ii[c]];
      v += t;
    }
    for (int d = 0; d < 3; ++d) {
      const int e = d == 0 ? 1 : 0, f = d == 2 ? 1 : 2;
      const double mm = a.M1[ii[e] * n + ii[e]] * a.M1[ii[f] * n + ii[f]] * a.h[e] * a.h[f] * a.coef;
      for (int s = 0; s < 2; ++s) {
        if (ii[d] != s * K) continue;  // phi vanishes on this face
        const bool has_nb = s == 1 ? cidx[d] + 1 < dims[d] : cidx[d] > 0;
        const bool dir_face = !has_nb && ((a.dmask >> (2 * d + s)) & 1u);
        if (!has_nb && !dir_face) continue;
        const double dphi = (s == 1 ? a.d1[ii[d]] : a.d0[ii[d]]) / a.h[d];  // d_{+d} phi / phi at the face
        if (has_nb) {
          // own "-" (s = 1): -phi d phi + sigma phi^2; own "+" (s = 0): +phi d phi + sigma phi^2
          v += mm * ((s == 1 ? -dphi : dphi) + a.sig_int[d]);
        } else {
          // -2 phi d_n phi + sigma_b phi^2, d_n = +-d_{+d}
          v += mm * ((s == 1 ? -2.0 * dphi : 2.0 * dphi) + a.sig_bnd[d]);
        }
      }
    }
    if (d64) d64[idx] = v;
    if (d32) d32[idx] = (float)v;
  }
}

static DgArgs dg_args(const mfx_op* op, const int32_t* skip) {
  DgArgs a{};
  const int n = op->n;
  a.nx = op->nx;
  a.ny = op->ny;
  a.nz = op->nz;
  a.n_cells = op->n_cells;
  for (int d = 0; d < 3; ++d) {
    a.h[d] = op->dg_h[d];
    a.sig_int[d] = op->dg_penalty * n * n / op->dg_h[d];
    a.sig_bnd[d] = op->dg_penalty * n * n * 2.0 / op->dg_h[d];
  }
  a.coef = op->dg_coef;
  a.dmask = op->dirichlet;
  const BasisTables& b = op->basis;
  for (int q = 0; q < n; ++q) a.wq[q] = b.wq[q];
  for (int i = 0; i < n * n; ++i) a.S[i] = b.S[i];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double k1 = 0.0, m1 = 0.0;
      for (int q = 0; q < n; ++q) {
        k1 += b.wq[q] * b.Sd[q * n + i] * b.Sd[q * n + j];
        m1 += b.wq[q] * b.S[q * n + i] * b.S[q * n + j];
      }
      a.K1[i * n + j] = k1;
      a.M1[i * n + j] = m1;
    }
  for (int i = 0; i < n; ++i) {
    a.d0[i] = lagrange_derivative(n, b.gll, i, 0.0);
    a.d1[i] = lagrange_derivative(n, b.gll, i, 1.0);
  }
  a.skip = skip;
  return a;
}

template <int N, typename Real>
static mfx_status run_dg(const mfx_op* op, const Real* src, Real* dst, cudaStream_t s, const int32_t* skip) {
  constexpr int N2 = N * N, N3 = N2 * N;
  constexpr int CB = 128 / N2 > 0 ? 128 / N2 : 1;
  const size_t smem = (size_t)CB * (5 * N3 + 6 * N2) * sizeof(Real);
  auto kern = dg_vmult_kernel<N, Real>;
  static int blocks_per_sm = -1;
  if (blocks_per_sm < 0) {
    MFX_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int b = 0;
    MFX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 128, smem));
    blocks_per_sm = b > 0 ? b : 1;
  }
  const DgArgs a = dg_args(op, skip);
  const int64_t nbatch = (op->n_cells + CB - 1) / CB;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(nbatch, (int64_t)device_sm_count() * blocks_per_sm));
  kern<<<grid, 128, smem, s>>>(a, src, dst);
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

template <typename Real>
static mfx_status dg_dispatch(const mfx_op* op, const Real* src, Real* dst, cudaStream_t s, const int32_t* skip) {
  switch (op->n) {
    case 2: return run_dg<2, Real>(op, src, dst, s, skip);
    case 3: return run_dg<3, Real>(op, src, dst, s, skip);
    case 4: return run_dg<4, Real>(op, src, dst, s, skip);
    case 5: return run_dg<5, Real>(op, src, dst, s, skip);
    case 6: return run_dg<6, Real>(op, src, dst, s, skip);
    case 7: return run_dg<7, Real>(op, src, dst, s, skip);
    case 8: return run_dg<8, Real>(op, src, dst, s, skip);
    case 9: return run_dg<9, Real>(op, src, dst, s, skip);
    default: return set_error(MFX_EUNSUPPORTED, "degree out of range");
  }
}

mfx_status launch_dg_vmult(const mfx_op* op, mfx_prec prec, const void* src, void* dst, cudaStream_t s,
                           const int32_t* skip) {
  if (prec == MFX_F64) return dg_dispatch<double>(op, (const double*)src, (double*)dst, s, skip);
  return dg_dispatch<float>(op, (const float*)src, (float*)dst, s, skip);
}

mfx_status launch_dg_diagonal(mfx_op* op, cudaStream_t s) {
  const DgArgs a = dg_args(op, nullptr);
  const int64_t total = op->n_dofs;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)device_sm_count() * 16));
  dg_diagonal_kernel<<<grid, 256, 0, s>>>(a, op->n, op->d_diag64, op->d_diag32);
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

}  // namespace mfx
