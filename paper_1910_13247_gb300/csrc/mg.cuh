// Geometric multigrid V-cycle (the paper's large-scale solver: conjugate gradients preconditioned by a
// multigrid V-cycle with Chebyshev smoothing and matrix-free transfers, Sec. 3.5, Sec. 6.1).
// Included at the end of solve.cu (it uses the solver's workspaces, Chebyshev and Lanczos code).
//
// Levels (structured boxes, same degree k): level l - 1 has half the cells per direction of level l;
// its vertices are every other vertex of level l's lattice.  Transfers between levels are matrix-free
// and sum-factorised: a coarse cell's Q_k values are interpolated to the (2k + 1)^3 fine lattice points
// inside it by three 1D sweeps with P1[i][j] = l_j(position of fine point i in the coarse cell), and
// restriction is the exact transpose.  Each fine point is owned by one coarse cell (the one below it in
// every direction, the last cell owning the far boundary), so prolongation writes every fine value once
// and restriction reads it once.  Dirichlet DoFs are masked on both sides.  The coarsest level is solved
// exactly with the inverse of its free-DoF block, formed once at set-up from operator applications to
// unit vectors and inverted on the host (Cholesky), then applied as a dense matrix-vector product.  All
// of a cycle is a fixed sequence of kernels on one stream, so it is captured with the PCG iterations.
//
// With an SIPG operator on top (the paper's DG benchmark hierarchy, Sec. 6.1), the top level is the
// discontinuous space on the finest mesh, reached from the continuous space of the same degree on the
// same mesh by injection (each DG node takes the continuous value at its lattice point, Dirichlet
// points 0); restriction is its transpose, a gather of the up to eight DG nodes on each lattice point.
// The DG level's vectors are flat (n_dofs x 1 x 1, nothing constrained).
#pragma once

#include <array>
#include <chrono>

namespace mfx {

constexpr int kMgMaxP = (2 * kMaxDegree + 1) * (kMaxDegree + 1);

struct MgLevel {
  mfx_mesh* mesh = nullptr;
  mfx_op* op = nullptr;
  int nx = 0, ny = 0, nz = 0, Mx = 0, My = 0, Mz = 0;
  uint32_t dmask = 0;
  bool dg = false;            // SIPG level (top of the hierarchy; flat vectors, no Dirichlet DoFs)
  double lo = 0.0, hi = 0.0;  // Chebyshev interval of the smoother
  double *b64 = nullptr, *x64 = nullptr, *r64 = nullptr, *c64 = nullptr;
  float *b32 = nullptr, *x32 = nullptr, *r32 = nullptr, *c32 = nullptr;
};

template <typename Real>
struct MgVec {
  static Real* b(MgLevel& L);
  static Real* x(MgLevel& L);
  static Real* r(MgLevel& L);
  static Real* c(MgLevel& L);
};
template <>
struct MgVec<double> {
  static double* b(MgLevel& L) { return L.b64; }
  static double* x(MgLevel& L) { return L.x64; }
  static double* r(MgLevel& L) { return L.r64; }
  static double* c(MgLevel& L) { return L.c64; }
};
template <>
struct MgVec<float> {
  static float* b(MgLevel& L) { return L.b32; }
  static float* x(MgLevel& L) { return L.x32; }
  static float* r(MgLevel& L) { return L.r32; }
  static float* c(MgLevel& L) { return L.c32; }
};

// Transfer between level c (coarse) and c + 1 (fine).
struct XferArgs {
  int nxc, nyc, nzc, Mxc, Myc, Mzc, Mxf, Myf, Mzf;
  uint32_t dmask_c, dmask_f;
  double P[kMgMaxP];  // (2k + 1) x (k + 1), row-major
  float P32[kMgMaxP];
};

template <typename Real>
__device__ __forceinline__ Real xfer_p(const XferArgs& a, int i) {
  if constexpr (sizeof(Real) == 8)
    return a.P[i];
  else
    return a.P32[i];
}

// xf += P xc on the cells' owned fine points (fine Dirichlet points untouched).  One CTA per coarse cell.
template <int N, typename Real>
__global__ void mg_prolongate_kernel(const __grid_constant__ XferArgs a, const Real* __restrict__ xc,
                                     Real* __restrict__ xf, const int32_t* skip) {
  constexpr int K = N - 1, F = 2 * K + 1;
  if (skip && *skip) return;
  __shared__ Real u[N * N * N], t1[F * N * N], t2[F * F * N];
  const int64_t cell = blockIdx.x;
  const int cx = (int)(cell % a.nxc);
  const int64_t rest = cell / a.nxc;
  const int cy = (int)(rest % a.nyc), cz = (int)(rest / a.nyc);
  for (int i = threadIdx.x; i < N * N * N; i += blockDim.x) {
    const int j1 = i % N, j2 = (i / N) % N, j3 = i / (N * N);
    const int I = cx * K + j1, J = cy * K + j2, L = cz * K + j3;
    u[i] = on_dirichlet(a.dmask_c, I, J, L, a.Mxc, a.Myc, a.Mzc)
               ? Real(0)
               : xc[(int64_t)I + (int64_t)a.Mxc * (J + (int64_t)a.Myc * L)];
  }
  __syncthreads();
  for (int l = threadIdx.x; l < N * N; l += blockDim.x) {  // along x: lines (j2, j3)
    for (int i1 = 0; i1 < F; ++i1) {
      Real s = Real(0);
#pragma unroll
      for (int j1 = 0; j1 < N; ++j1) s += xfer_p<Real>(a, i1 * N + j1) * u[j1 + N * l];
      t1[i1 + F * l] = s;
    }
  }
  __syncthreads();
  for (int l = threadIdx.x; l < F * N; l += blockDim.x) {  // along y: lines (i1, j3)
    const int i1 = l % F, j3 = l / F;
    for (int i2 = 0; i2 < F; ++i2) {
      Real s = Real(0);
#pragma unroll
      for (int j2 = 0; j2 < N; ++j2) s += xfer_p<Real>(a, i2 * N + j2) * t1[i1 + F * (j2 + N * j3)];
      t2[i1 + F * (i2 + F * j3)] = s;
    }
  }
  __syncthreads();
  for (int l = threadIdx.x; l < F * F; l += blockDim.x) {  // along z: lines (i1, i2), written out
    const int i1 = l % F, i2 = l / F;
    const int I = cx * 2 * K + i1, J = cy * 2 * K + i2;
    if ((i1 == 2 * K && cx != a.nxc - 1) || (i2 == 2 * K && cy != a.nyc - 1)) continue;
    for (int i3 = 0; i3 < F; ++i3) {
      if (i3 == 2 * K && cz != a.nzc - 1) continue;
      const int L = cz * 2 * K + i3;
      if (on_dirichlet(a.dmask_f, I, J, L, a.Mxf, a.Myf, a.Mzf)) continue;
      Real s = Real(0);
#pragma unroll
      for (int j3 = 0; j3 < N; ++j3) s += xfer_p<Real>(a, i3 * N + j3) * t2[i1 + F * (i2 + F * j3)];
      xf[(int64_t)I + (int64_t)a.Mxf * (J + (int64_t)a.Myf * L)] += s;
    }
  }
}

// bc += P^T rf over the cells' owned fine points (coarse Dirichlet points untouched).
template <int N, typename Real>
__global__ void mg_restrict_kernel(const __grid_constant__ XferArgs a, const Real* __restrict__ rf,
                                   Real* __restrict__ bc, const int32_t* skip) {
  constexpr int K = N - 1, F = 2 * K + 1;
  if (skip && *skip) return;
  __shared__ Real t2[F * F * N], t1[F * N * N];
  const int64_t cell = blockIdx.x;
  const int cx = (int)(cell % a.nxc);
  const int64_t rest = cell / a.nxc;
  const int cy = (int)(rest % a.nyc), cz = (int)(rest / a.nyc);
  for (int l = threadIdx.x; l < F * F; l += blockDim.x) {  // along z from the owned fine points
    const int i1 = l % F, i2 = l / F;
    const int I = cx * 2 * K + i1, J = cy * 2 * K + i2;
    const bool own12 = !((i1 == 2 * K && cx != a.nxc - 1) || (i2 == 2 * K && cy != a.nyc - 1));
    Real f[F];
    for (int i3 = 0; i3 < F; ++i3) {
      const int L = cz * 2 * K + i3;
      const bool own = own12 && !(i3 == 2 * K && cz != a.nzc - 1) &&
                       !on_dirichlet(a.dmask_f, I, J, L, a.Mxf, a.Myf, a.Mzf);
      f[i3] = own ? rf[(int64_t)I + (int64_t)a.Mxf * (J + (int64_t)a.Myf * L)] : Real(0);
    }
#pragma unroll
    for (int j3 = 0; j3 < N; ++j3) {
      Real s = Real(0);
      for (int i3 = 0; i3 < F; ++i3) s += xfer_p<Real>(a, i3 * N + j3) * f[i3];
      t2[i1 + F * (i2 + F * j3)] = s;
    }
  }
  __syncthreads();
  for (int l = threadIdx.x; l < F * N; l += blockDim.x) {  // along y: lines (i1, j3)
    const int i1 = l % F, j3 = l / F;
#pragma unroll
    for (int j2 = 0; j2 < N; ++j2) {
      Real s = Real(0);
      for (int i2 = 0; i2 < F; ++i2) s += xfer_p<Real>(a, i2 * N + j2) * t2[i1 + F * (i2 + F * j3)];
      t1[i1 + F * (j2 + N * j3)] = s;
    }
  }
  __syncthreads();
  for (int l = threadIdx.x; l < N * N; l += blockDim.x) {  // along x: lines (j2, j3), added in
    const int j2 = l % N, j3 = l / N;
    const int J = cy * K + j2, L = cz * K + j3;
#pragma unroll
    for (int j1 = 0; j1 < N; ++j1) {
      const int I = cx * K + j1;
      if (on_dirichlet(a.dmask_c, I, J, L, a.Mxc, a.Myc, a.Mzc)) continue;
      Real s = Real(0);
      for (int i1 = 0; i1 < F; ++i1) s += xfer_p<Real>(a, i1 * N + j1) * t1[i1 + F * (j2 + N * j3)];
      atomicAdd(bc + (int64_t)I + (int64_t)a.Mxc * (J + (int64_t)a.Myc * L), s);
    }
  }
}

// Injection of the continuous level c into the DG level f on the same cells: xf[c n^3 + i] += xc at the
// lattice point of cell c's node i (nothing for Dirichlet points).  One thread per DG DoF.
template <typename Real>
__global__ void mg_inject_kernel(const __grid_constant__ XferArgs a, int n, const Real* __restrict__ xc,
                                 Real* __restrict__ xf, const int32_t* skip) {
  if (skip && *skip) return;
  const int k = n - 1, n3 = n * n * n;
  const int64_t total = (int64_t)a.nxc * a.nyc * a.nzc * n3;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = idx / n3;
    const int i = (int)(idx - cell * n3);
    const int64_t I = (cell % a.nxc) * k + i % n;
    const int64_t J = ((cell / a.nxc) % a.nyc) * k + (i / n) % n;
    const int64_t L = (cell / ((int64_t)a.nxc * a.nyc)) * k + i / (n * n);
    if (!on_dirichlet(a.dmask_c, I, J, L, a.Mxc, a.Myc, a.Mzc)) xf[idx] += xc[I + a.Mxc * (J + (int64_t)a.Myc * L)];
  }
}

// Transpose of the injection: xc[p] += sum of xf over the DG nodes at lattice point p (free p only).
// Along one direction a lattice index I is node I mod k of cell I / k, or, where I is a multiple of k,
// node k of cell I / k - 1 and node 0 of cell I / k (those that exist).  One thread per lattice point.
template <typename Real>
__global__ void mg_inject_t_kernel(const __grid_constant__ XferArgs a, int n, const Real* __restrict__ xf,
                                   Real* __restrict__ xc, const int32_t* skip) {
  if (skip && *skip) return;
  const int k = n - 1, n3 = n * n * n;
  const int64_t total = (int64_t)a.Mxc * a.Myc * a.Mzc;
  const int nc[3] = {a.nxc, a.nyc, a.nzc};
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = p % a.Mxc, rest = p / a.Mxc, J = rest % a.Myc, L = rest / a.Myc;
    if (on_dirichlet(a.dmask_c, I, J, L, a.Mxc, a.Myc, a.Mzc)) continue;
    const int64_t lat[3] = {I, J, L};
    int cnt[3], cc[3][2], ci[3][2];
    for (int d = 0; d < 3; ++d) {
      const int c = (int)(lat[d] / k), r = (int)(lat[d] - (int64_t)c * k);
      cnt[d] = 0;
      if (r == 0 && c > 0) {
        cc[d][cnt[d]] = c - 1;
        ci[d][cnt[d]++] = k;
      }
      if (c < nc[d]) {
        cc[d][cnt[d]] = c;
        ci[d][cnt[d]++] = r;
      }
    }
    Real s = Real(0);
    for (int c3 = 0; c3 < cnt[2]; ++c3)
      for (int c2 = 0; c2 < cnt[1]; ++c2)
        for (int c1 = 0; c1 < cnt[0]; ++c1) {
          const int64_t cell = cc[0][c1] + (int64_t)nc[0] * (cc[1][c2] + (int64_t)nc[1] * cc[2][c3]);
          s += xf[cell * n3 + ci[0][c1] + n * (ci[1][c2] + n * ci[2][c3])];
        }
    xc[p] += s;
  }
}

// out = (in1 - in2) on free DoFs (in2 may be null: out = in1), 0 on Dirichlet DoFs.
template <typename Real>
__global__ void mg_masked_diff_kernel(int Mx, int My, int Mz, uint32_t dmask, const Real* __restrict__ in1,
                                      const Real* __restrict__ in2, Real* __restrict__ out, const int32_t* skip) {
  if (skip && *skip) return;
  const int64_t n = (int64_t)Mx * My * Mz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = i % Mx, rest = i / Mx, J = rest % My, L = rest / My;
    out[i] = on_dirichlet(dmask, I, J, L, Mx, My, Mz) ? Real(0) : (in2 ? in1[i] - in2[i] : in1[i]);
  }
}

// z = x on free DoFs, r on Dirichlet DoFs (the identity block of the condensed operator); or x += y.
template <typename Real>
__global__ void mg_finish_kernel(int Mx, int My, int Mz, uint32_t dmask, const Real* __restrict__ x,
                                 const Real* __restrict__ r, Real* __restrict__ z, const int32_t* skip) {
  if (skip && *skip) return;
  const int64_t n = (int64_t)Mx * My * Mz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = i % Mx, rest = i / Mx, J = rest % My, L = rest / My;
    z[i] = on_dirichlet(dmask, I, J, L, Mx, My, Mz) ? r[i] : x[i];
  }
}
template <typename Real>
__global__ void mg_axpy_kernel(int64_t n, Real* __restrict__ x, const Real* __restrict__ y, const int32_t* skip) {
  if (skip && *skip) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += y[i];
}

// Coarse solve: x[free[i]] = sum_j inv[i][j] b[free[j]]; one warp per row (x zeroed before).
template <typename Real>
__global__ void mg_coarse_kernel(int nf, const int32_t* __restrict__ free, const Real* __restrict__ inv,
                                 const Real* __restrict__ b, Real* __restrict__ x, const int32_t* skip) {
  if (skip && *skip) return;
  const int lane = threadIdx.x & 31;
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < nf; row += (gridDim.x * blockDim.x) >> 5) {
    const Real* a = inv + (int64_t)row * nf;
    Real s = Real(0);
    for (int j = lane; j < nf; j += 32) s += a[j] * b[free[j]];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) x[free[row]] = s;
  }
}

// e_j on the free DoF free[j] (all else 0)
__global__ void mg_unit_kernel(int64_t n, int64_t dof, double* __restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = i == dof ? 1.0 : 0.0;
}
__global__ void mg_gather_col_kernel(int nf, const int32_t* __restrict__ free, const double* __restrict__ y,
                                     double* __restrict__ col) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) col[i] = y[free[i]];
}
__global__ void mg_fill_kernel(int Mx, int My, int Mz, uint32_t dmask, double* __restrict__ v) {
  const int64_t n = (int64_t)Mx * My * Mz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = i % Mx, rest = i / Mx, J = rest % My, L = rest / My;
    v[i] = on_dirichlet(dmask, I, J, L, Mx, My, Mz) ? 0.0 : 1.0;
  }
}

}  // namespace mfx

struct mfx_mg {
  std::vector<mfx::MgLevel> levels;  // coarse to fine
  std::vector<mfx::XferArgs> xfer;   // xfer[l]: level l - 1 to level l (xfer[0] unused)
  int k = 0, degree = 6;
  bool has_f32 = false;
  int nf = 0;                        // free DoFs of the coarsest level
  int32_t* d_free = nullptr;
  double* d_inv64 = nullptr;
  float* d_inv32 = nullptr;
  void* d_vecs = nullptr;            // all level vectors (one stream-ordered allocation)
  cudaStream_t stream = nullptr;     // set-up stream
};

namespace mfx {

template <typename Real>
static mfx_status mg_transfer(mfx_mg* mg, int l, bool prolong, const Real* in, Real* out, const int32_t* skip,
                              cudaStream_t s) {
  const XferArgs& a = mg->xfer[l];
  if (mg->levels[l].dg) {
    const int n = mg->k + 1;
    const int64_t work = prolong ? mg->levels[l].op->n_dofs : (int64_t)a.Mxc * a.Myc * a.Mzc;
    if (prolong)
      mg_inject_kernel<Real><<<vec_grid(work), 256, 0, s>>>(a, n, in, out, skip);
    else
      mg_inject_t_kernel<Real><<<vec_grid(work), 256, 0, s>>>(a, n, in, out, skip);
    MFX_CUDA_TRY(cudaGetLastError());
    return MFX_OK;
  }
  const unsigned cells = (unsigned)((int64_t)a.nxc * a.nyc * a.nzc);
  const int F = 2 * mg->k + 1;
  const int threads = std::min(256, std::max(32, (F * F + 31) / 32 * 32));
#define MFX_MG_CASE(NN)                                                                                 \
  case NN:                                                                                              \
    if (prolong)                                                                                        \
      mg_prolongate_kernel<NN, Real><<<cells, threads, 0, s>>>(a, in, out, skip);                        \
    else                                                                                                \
      mg_restrict_kernel<NN, Real><<<cells, threads, 0, s>>>(a, in, out, skip);                          \
    break;
  switch (mg->k + 1) {
    MFX_MG_CASE(2) MFX_MG_CASE(3) MFX_MG_CASE(4) MFX_MG_CASE(5) MFX_MG_CASE(6) MFX_MG_CASE(7) MFX_MG_CASE(8)
    MFX_MG_CASE(9)
    default: return set_error(MFX_EUNSUPPORTED, "multigrid degree");
  }
#undef MFX_MG_CASE
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

// The cycle on level l for K_l x_l = b_l (level vectors), as the oracle writes it.
template <typename Real>
static mfx_status mg_cycle(mfx_mg* mg, int l, const int32_t* skip, cudaStream_t s) {
  MgLevel& L = mg->levels[l];
  Real* b = MgVec<Real>::b(L);
  Real* x = MgVec<Real>::x(L);
  const int64_t n = L.op->n_dofs;
  if (l == 0) {
    MFX_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(Real) * n, s));
    const Real* inv = std::is_same<Real, double>::value ? (const Real*)mg->d_inv64 : (const Real*)mg->d_inv32;
    if (mg->nf > 0)
      mg_coarse_kernel<Real><<<std::max(1, std::min((mg->nf + 7) / 8, 4 * device_sm_count())), 256, 0, s>>>(
          mg->nf, mg->d_free, inv, b, x, skip);
    MFX_CUDA_TRY(cudaGetLastError());
    return MFX_OK;
  }
  Real* res = MgVec<Real>::r(L);
  Real* corr = MgVec<Real>::c(L);
  Work<Real>& w = work_of<Real>(workspace(L.op));
  MgLevel& C = mg->levels[l - 1];
  // pre-smoothing from zero
  mfx_status rc = cheb_apply<Real>(L.op, w, b, x, mg->degree, L.lo, L.hi, skip, s);
  if (rc != MFX_OK) return rc;
  // coarse correction
  rc = launch_vmult(L.op, prec_of<Real>(), x, w.t, s, skip);
  if (rc != MFX_OK) return rc;
  mg_masked_diff_kernel<Real><<<vec_grid(n), 256, 0, s>>>(L.Mx, L.My, L.Mz, L.dmask, b, w.t, res, skip);
  MFX_CUDA_TRY(cudaMemsetAsync(MgVec<Real>::b(C), 0, sizeof(Real) * C.op->n_dofs, s));
  rc = mg_transfer<Real>(mg, l, false, res, MgVec<Real>::b(C), skip, s);
  if (rc != MFX_OK) return rc;
  rc = mg_cycle<Real>(mg, l - 1, skip, s);
  if (rc != MFX_OK) return rc;
  rc = mg_transfer<Real>(mg, l, true, MgVec<Real>::x(C), x, skip, s);
  if (rc != MFX_OK) return rc;
  // post-smoothing
  rc = launch_vmult(L.op, prec_of<Real>(), x, w.t, s, skip);
  if (rc != MFX_OK) return rc;
  mg_masked_diff_kernel<Real><<<vec_grid(n), 256, 0, s>>>(L.Mx, L.My, L.Mz, L.dmask, b, w.t, res, skip);
  rc = cheb_apply<Real>(L.op, w, res, corr, mg->degree, L.lo, L.hi, skip, s);
  if (rc != MFX_OK) return rc;
  mg_axpy_kernel<Real><<<vec_grid(n), 256, 0, s>>>(n, x, corr, skip);
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

template <typename Real>
mfx_status mg_vcycle(mfx_mg* mg, const Real* r, Real* z, const int32_t* skip, cudaStream_t s) {
  if (!mg) return set_error(MFX_EINVAL, "no multigrid hierarchy");
  if (std::is_same<Real, float>::value && !mg->has_f32) return set_error(MFX_EINVAL, "multigrid has no FP32 data");
  const int top = (int)mg->levels.size() - 1;
  MgLevel& F = mg->levels[top];
  const int64_t n = F.op->n_dofs;
  mg_masked_diff_kernel<Real><<<vec_grid(n), 256, 0, s>>>(F.Mx, F.My, F.Mz, F.dmask, r, nullptr, MgVec<Real>::b(F),
                                                          skip);
  mfx_status rc = mg_cycle<Real>(mg, top, skip, s);
  if (rc != MFX_OK) return rc;
  mg_finish_kernel<Real><<<vec_grid(n), 256, 0, s>>>(F.Mx, F.My, F.Mz, F.dmask, MgVec<Real>::x(F), r, z, skip);
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

static void mg_free(mfx_mg* mg) {
  if (!mg) return;
  if (mg->stream) cudaStreamSynchronize(mg->stream);
  for (auto& L : mg->levels) {
    if (L.op) mfx_operator_destroy(L.op);
    if (L.mesh) mfx_mesh_destroy(L.mesh);
  }
  cudaStream_t s = mg->stream ? mg->stream : cudaStreamPerThread;
  if (mg->d_vecs) cudaFreeAsync(mg->d_vecs, s);
  if (mg->d_free) cudaFreeAsync(mg->d_free, s);
  if (mg->d_inv64) cudaFreeAsync(mg->d_inv64, s);
  if (mg->d_inv32) cudaFreeAsync(mg->d_inv32, s);
  cudaStreamSynchronize(s);
  if (mg->stream) cudaStreamDestroy(mg->stream);
  delete mg;
}

// Inverse of an SPD matrix (row-major, n x n) by Cholesky: A = L L^T, A^-1 = L^-T L^-1.
static bool spd_inverse(std::vector<double>& A, int n) {
  std::vector<double> L((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double d = A[(size_t)j * n + j];
    for (int p = 0; p < j; ++p) d -= L[(size_t)j * n + p] * L[(size_t)j * n + p];
    if (!(d > 0.0)) return false;
    const double ljj = std::sqrt(d);
    L[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double v = A[(size_t)i * n + j];
      for (int p = 0; p < j; ++p) v -= L[(size_t)i * n + p] * L[(size_t)j * n + p];
      L[(size_t)i * n + j] = v / ljj;
    }
  }
  // Linv (lower triangular)
  std::vector<double> Li((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    Li[(size_t)j * n + j] = 1.0 / L[(size_t)j * n + j];
    for (int i = j + 1; i < n; ++i) {
      double v = 0.0;
      for (int p = j; p < i; ++p) v -= L[(size_t)i * n + p] * Li[(size_t)p * n + j];
      Li[(size_t)i * n + j] = v / L[(size_t)i * n + i];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double v = 0.0;
      for (int p = i; p < n; ++p) v += Li[(size_t)p * n + i] * Li[(size_t)p * n + j];
      A[(size_t)i * n + j] = v;
      A[(size_t)j * n + i] = v;
    }
  return true;
}

}  // namespace mfx

extern "C" {

void mfx_mg_params_default(mfx_mg_params* p) {
  if (!p) return;
  *p = mfx_mg_params{};
  p->max_levels = 0;
  p->smoother_degree = 6;
  p->smoothing_range = 20.0;
  p->lanczos_steps = 15;
}

mfx_status mfx_mg_create(mfx_mg** out, const mfx_mesh* mesh, const mfx_op_desc* desc, const mfx_mg_params* params,
                         mfx_stream stream) try {
  MFX_TRACE("mfx_mg_create");
  if (!out || !mesh || !desc) return set_error(MFX_EINVAL, "mfx_mg_create: null argument");
  *out = nullptr;
  const Mesh& fm = mesh->m;
  if (!fm.structured) return set_error(MFX_EUNSUPPORTED, "multigrid levels need a structured mesh");
  if (desc->coef_kind == MFX_COEF_QPOINT)
    return set_error(MFX_EUNSUPPORTED, "multigrid: per-quadrature-point coefficients exist on one level only");
  const bool dg_top = desc->discretization == MFX_SIPG;
  if (dg_top && desc->coef_kind != MFX_COEF_CONSTANT)
    return set_error(MFX_EUNSUPPORTED, "SIPG takes a constant coefficient");
  mfx_op_desc cg_desc = *desc;  // the continuous levels
  cg_desc.discretization = MFX_CONTINUOUS;
  mfx_mg_params p;
  mfx_mg_params_default(&p);
  if (params) p = *params;
  if (p.smoother_degree < 1 || !(p.smoothing_range > 1.0) || p.lanczos_steps < 2 || p.max_levels < 0)
    return set_error(MFX_EINVAL, "mfx_mg_create: bad parameters");
  // level sizes: halve while all three counts are even (a 2:1:1 box of 2^(l+1) x 2^l x 2^l cells ends on
  // 2 x 1 x 1 cells, the coarse mesh of the paper's benchmark, Sec. 6.1)
  std::vector<std::array<int, 3>> sizes = {{fm.nx, fm.ny, fm.nz}};
  while (sizes.front()[0] % 2 == 0 && sizes.front()[1] % 2 == 0 && sizes.front()[2] % 2 == 0 &&
         (p.max_levels == 0 || (int)sizes.size() < p.max_levels))
    sizes.insert(sizes.begin(), {sizes.front()[0] / 2, sizes.front()[1] / 2, sizes.front()[2] / 2});
  auto* mg = new (std::nothrow) mfx_mg();
  if (!mg) return set_error(MFX_ENOMEM, "host allocation failed");
  mg->k = desc->degree;
  mg->degree = p.smoother_degree;
  mg->has_f32 = (desc->precisions == 0 || (desc->precisions & 2));
  const int ncg = (int)sizes.size();
  const int nl = ncg + (dg_top ? 1 : 0);
  mg->levels.resize(nl);
  mg->xfer.resize(nl);
  cudaStream_t s = (cudaStream_t)stream;
  auto fail = [&](mfx_status st) {
    mg_free(mg);
    return st;
  };
  if (cudaStreamCreateWithFlags(&mg->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(cuda_error(cudaErrorUnknown, "mg stream"));
  MFX_CUDA_TRY(cudaStreamSynchronize(s));
  // meshes: the finest is a copy of the caller's; each coarser one takes every other vertex
  std::vector<double> verts = fm.vertices;
  for (int l = ncg - 1; l >= 0; --l) {
    MgLevel& L = mg->levels[l];
    L.nx = sizes[l][0];
    L.ny = sizes[l][1];
    L.nz = sizes[l][2];
    if (l < ncg - 1) {
      const int fx = sizes[l + 1][0], fy = sizes[l + 1][1];
      std::vector<double> c((size_t)3 * (L.nx + 1) * (L.ny + 1) * (L.nz + 1));
      for (int kz = 0; kz <= L.nz; ++kz)
        for (int jy = 0; jy <= L.ny; ++jy)
          for (int ix = 0; ix <= L.nx; ++ix)
            for (int d = 0; d < 3; ++d)
              c[3 * ((size_t)ix + (L.nx + 1) * ((size_t)jy + (L.ny + 1) * kz)) + d] =
                  verts[3 * ((size_t)2 * ix + (fx + 1) * ((size_t)2 * jy + (fy + 1) * (size_t)2 * kz)) + d];
      verts.swap(c);
    }
    mfx_status st = mfx_mesh_create_structured(&L.mesh, L.nx, L.ny, L.nz, verts.data());
    if (st != MFX_OK) return fail(st);
    L.mesh->m.dirichlet = fm.dirichlet;
    st = mfx_operator_create(&L.op, L.mesh, &cg_desc, (mfx_stream)mg->stream);
    if (st != MFX_OK) return fail(st);
    st = ensure_workspace(L.op);
    if (st != MFX_OK) return fail(st);
    L.Mx = mg->k * L.nx + 1;
    L.My = mg->k * L.ny + 1;
    L.Mz = mg->k * L.nz + 1;
    L.dmask = fm.dirichlet;
  }
  if (dg_top) {  // the SIPG operator of the caller's mesh
    MgLevel& L = mg->levels[ncg];
    L.dg = true;
    L.nx = fm.nx;
    L.ny = fm.ny;
    L.nz = fm.nz;
    mfx_status st = mfx_operator_create(&L.op, mesh, desc, (mfx_stream)mg->stream);
    if (st != MFX_OK) return fail(st);
    st = ensure_workspace(L.op);
    if (st != MFX_OK) return fail(st);
    L.Mx = (int)L.op->n_dofs;
    L.My = L.Mz = 1;
    L.dmask = 0;
  }
  // level vectors
  size_t total = 0;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  for (auto& L : mg->levels) total += 4 * al(sizeof(double) * L.op->n_dofs) + (mg->has_f32 ? 4 * al(sizeof(float) * L.op->n_dofs) : 0);
  if (cudaMallocAsync(&mg->d_vecs, total, mg->stream) != cudaSuccess) return fail(set_error(MFX_ENOMEM, "multigrid vectors"));
  char* q = (char*)mg->d_vecs;
  for (auto& L : mg->levels) {
    const size_t b64 = al(sizeof(double) * L.op->n_dofs), b32 = al(sizeof(float) * L.op->n_dofs);
    double** v64[] = {&L.b64, &L.x64, &L.r64, &L.c64};
    for (auto* v : v64) {
      *v = (double*)q;
      q += b64;
    }
    if (mg->has_f32) {
      float** v32[] = {&L.b32, &L.x32, &L.r32, &L.c32};
      for (auto* v : v32) {
        *v = (float*)q;
        q += b32;
      }
    }
  }
  // transfers: P1[i][j] = l_j(position of fine lattice point i of a coarse cell)
  BasisTables bt;
  make_basis(mg->k, &bt);
  const int K = mg->k, N = K + 1, F = 2 * K + 1;
  std::vector<double> gll(N);
  for (int j = 0; j < N; ++j) gll[j] = bt.gll[j];
  for (int l = 1; l < nl; ++l) {
    XferArgs& a = mg->xfer[l];
    const MgLevel &C = mg->levels[l - 1], &Fl = mg->levels[l];
    a.nxc = C.nx;
    a.nyc = C.ny;
    a.nzc = C.nz;
    a.Mxc = C.Mx;
    a.Myc = C.My;
    a.Mzc = C.Mz;
    a.Mxf = Fl.Mx;
    a.Myf = Fl.My;
    a.Mzf = Fl.Mz;
    a.dmask_c = C.dmask;
    a.dmask_f = Fl.dmask;
    if (Fl.dg) continue;  // injection: no interpolation table
    for (int i = 0; i < F; ++i) {
      const double pos = i <= K ? gll[i] / 2.0 : (1.0 + gll[i - K]) / 2.0;
      for (int j = 0; j < N; ++j) {
        const double v = lagrange_value(N, gll.data(), j, pos);
        a.P[i * N + j] = v;
        a.P32[i * N + j] = (float)v;
      }
    }
  }
  // smoother intervals from Lanczos on each level (start: ones on the free DoFs)
  for (int l = 1; l < nl; ++l) {
    MgLevel& L = mg->levels[l];
    mg_fill_kernel<<<vec_grid(L.op->n_dofs), 256, 0, mg->stream>>>(L.Mx, L.My, L.Mz, L.dmask, L.r64);
    double lam = 0.0;
    mfx_status st = estimate_lambda<double>(L.op, workspace(L.op), L.r64, p.lanczos_steps, mg->stream, &lam);
    if (st != MFX_OK) return fail(st);
    L.hi = 1.2 * lam;
    L.lo = L.hi / p.smoothing_range;
  }
  // coarsest level: inverse of the free block from K e_j
  {
    MgLevel& C = mg->levels[0];
    std::vector<int32_t> free;
    for (int64_t i = 0; i < C.op->n_dofs; ++i) {
      const int64_t I = i % C.Mx, rest = i / C.Mx, J = rest % C.My, Lz = rest / C.My;
      if (!on_dirichlet(C.dmask, I, J, Lz, C.Mx, C.My, C.Mz)) free.push_back((int32_t)i);
    }
    const int nf = (int)free.size();
    if (nf > 8192) return fail(set_error(MFX_EUNSUPPORTED, "coarsest multigrid level too large for a dense solve"));
    mg->nf = nf;
    if (nf > 0) {
      double* col = nullptr;
      if (cudaMallocAsync((void**)&mg->d_free, sizeof(int32_t) * nf, mg->stream) != cudaSuccess ||
          cudaMallocAsync((void**)&mg->d_inv64, sizeof(double) * nf * nf, mg->stream) != cudaSuccess ||
          cudaMallocAsync((void**)&col, sizeof(double) * nf * nf, mg->stream) != cudaSuccess)
        return fail(set_error(MFX_ENOMEM, "coarse matrix"));
      MFX_CUDA_TRY(cudaMemcpyAsync(mg->d_free, free.data(), sizeof(int32_t) * nf, cudaMemcpyHostToDevice, mg->stream));
      for (int j = 0; j < nf; ++j) {
        mg_unit_kernel<<<vec_grid(C.op->n_dofs), 256, 0, mg->stream>>>(C.op->n_dofs, free[j], C.x64);
        mfx_status st = launch_vmult(C.op, MFX_F64, C.x64, C.r64, mg->stream);
        if (st != MFX_OK) return fail(st);
        mg_gather_col_kernel<<<(nf + 255) / 256, 256, 0, mg->stream>>>(nf, mg->d_free, C.r64, col + (size_t)j * nf);
      }
      std::vector<double> A((size_t)nf * nf);
      MFX_CUDA_TRY(cudaMemcpyAsync(A.data(), col, sizeof(double) * nf * nf, cudaMemcpyDeviceToHost, mg->stream));
      MFX_CUDA_TRY(cudaStreamSynchronize(mg->stream));
      cudaFreeAsync(col, mg->stream);
      // symmetrise against rounding of the column-wise products, then invert
      for (int i = 0; i < nf; ++i)
        for (int j = 0; j < i; ++j) {
          const double v = 0.5 * (A[(size_t)i * nf + j] + A[(size_t)j * nf + i]);
          A[(size_t)i * nf + j] = A[(size_t)j * nf + i] = v;
        }
      if (!spd_inverse(A, nf)) return fail(set_error(MFX_EINVAL, "coarse operator is not positive definite"));
      MFX_CUDA_TRY(cudaMemcpyAsync(mg->d_inv64, A.data(), sizeof(double) * nf * nf, cudaMemcpyHostToDevice, mg->stream));
      if (mg->has_f32) {
        std::vector<float> A32(A.begin(), A.end());
        if (cudaMallocAsync((void**)&mg->d_inv32, sizeof(float) * nf * nf, mg->stream) != cudaSuccess)
          return fail(set_error(MFX_ENOMEM, "coarse matrix"));
        MFX_CUDA_TRY(cudaMemcpyAsync(mg->d_inv32, A32.data(), sizeof(float) * nf * nf, cudaMemcpyHostToDevice, mg->stream));
        MFX_CUDA_TRY(cudaStreamSynchronize(mg->stream));
      }
    }
  }
  MFX_CUDA_TRY(cudaStreamSynchronize(mg->stream));
  *out = mg;
  return MFX_OK;
} catch (...) {
  return host_exception();
}

void mfx_mg_destroy(mfx_mg* mg) { mg_free(mg); }

mfx_status mfx_mg_info(const mfx_mg* mg, int32_t* n_levels, int32_t* coarse_free_dofs) {
  if (!mg) return set_error(MFX_EINVAL, "null multigrid");
  if (n_levels) *n_levels = (int32_t)mg->levels.size();
  if (coarse_free_dofs) *coarse_free_dofs = mg->nf;
  return MFX_OK;
}

const mfx_op* mfx_mg_operator(const mfx_mg* mg, int32_t level) {
  if (!mg || level < 0 || level >= (int32_t)mg->levels.size()) return nullptr;
  return mg->levels[level].op;
}

mfx_status mfx_mg_get_bounds(const mfx_mg* mg, int32_t level, double* lo, double* hi) {
  if (!mg || !lo || !hi || level < 0 || level >= (int32_t)mg->levels.size()) return set_error(MFX_EINVAL, "bad level");
  *lo = mg->levels[level].lo;
  *hi = mg->levels[level].hi;
  return MFX_OK;
}

mfx_status mfx_mg_set_bounds(mfx_mg* mg, int32_t level, double lo, double hi) {
  if (!mg || level < 1 || level >= (int32_t)mg->levels.size() || !(lo > 0.0) || !(hi > lo))
    return set_error(MFX_EINVAL, "bad level or interval");
  mg->levels[level].lo = lo;
  mg->levels[level].hi = hi;
  return MFX_OK;
}

mfx_status mfx_mg_vcycle(mfx_mg* mg, mfx_prec prec, const void* r, void* z, mfx_stream stream) {
  if (!mg || !r || !z || r == z) return set_error(MFX_EINVAL, "mfx_mg_vcycle: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == MFX_F64) return mg_vcycle<double>(mg, (const double*)r, (double*)z, nullptr, s);
  if (prec == MFX_F32) return mg_vcycle<float>(mg, (const float*)r, (float*)z, nullptr, s);
  return set_error(MFX_EINVAL, "mfx_mg_vcycle: precision");
}

mfx_status mfx_mg_solve(mfx_mg* mg, const double* b, double* x, const mfx_solve_params* params,
                        mfx_solve_stats* stats, mfx_stream stream) {
  MFX_TRACE("mfx_mg_solve");
  if (!mg) return set_error(MFX_EINVAL, "null multigrid");
  return solve_impl(mg->levels.back().op, b, x, params, mg, stats, stream);
}

}  // extern "C"
