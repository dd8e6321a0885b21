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
// On a uniform Cartesian mesh with a constant coefficient the operator is a sum of Kronecker products,
//   A = a sum_d  L_d (x) (h_e M1) (x) (h_f M1)      (e, f the other two directions),
// with M1 the exact 1D mass matrix of the nodal basis on [0, 1] (n-point Gauss is exact for it) and L_d
// the 1D SIPG matrix along direction d: per cell K1 / h_d (K1 the 1D stiffness on [0, 1]) plus, at each
// cell end, rank-two face terms in the end value and end derivative of the cell's own line and of the
// neighbour's line across that end.  With GLL nodes the end value is the end node, so for a line x of a
// cell (l_j the 1D basis, d0_j = l_j'(0), d1_j = l_j'(1), K = n - 1, f = 1/2 at interior ends, 1 at
// Dirichlet ends, 0 at natural ends, sigma the end's penalty, w the neighbour's line):
//   lower end:  (L x)_i += f (delta_i0 g0 + d0_i x_0 / h) + sigma delta_i0 x_0,   g0 = sum_j d0_j x_j / h
//      interior also:  += delta_i0 gw / 2 - d0_i w_K / (2h) - sigma delta_i0 w_K, gw = sum_j d1_j w_j / h
//   upper end:  (L x)_i += -f (delta_iK g1 + d1_i x_K / h) + sigma delta_iK x_K,  g1 = sum_j d1_j x_j / h
//      interior also:  += -delta_iK gw / 2 + d1_i w_0 / (2h) - sigma delta_iK w_0, gw = sum_j d0_j w_j / h
// (the SIPG face integrals of one direction; their tangential factors are the tangential mass matrices).
//
// Element-centric: a CTA takes CB cells (one contiguous chunk of DoFs, staged in shared memory by
// coalesced loads), one thread per line of a cell, and writes each cell's output block once, without
// atomics.  Per cell, with the tangential masses shared between directions:
//   P = L_x u, Q = L_y u, R = L_z u          (1D SIPG sweeps; the neighbours' lines from global memory)
//   T1 = M_y P, T2 = M_x Q, T3 = M_x R
//   y = M_z (T1 + T2) + M_y T3               (eight sweeps, three barriers per batch of cells)
// The 1D tables are compile-time-indexed kernel parameters in the kernel's own precision, so the
// contractions read them as constant-bank operands.
#include <algorithm>

#include "basis_tables.h"
#include "df.cuh"
#include "mfx_internal.h"

namespace mfx {

int device_sm_count();

struct DgArgs {
  int nx, ny, nz;
  int64_t n_cells;
  double h[3], hinv[3];
  double coef, sig_int[3], sig_bnd[3];
  double scale[3];  // a h_e h_f: the factor of direction d's term
  uint32_t dmask;
  // 1D tables (n <= 9): K1, M1 (n x n, row-major), end derivatives l_i'(0), l_i'(1)
  double K1[kMaxN * kMaxN], M1[kMaxN * kMaxN], d0[kMaxN], d1[kMaxN];
  float K1f[kMaxN * kMaxN], M1f[kMaxN * kMaxN], d0f[kMaxN], d1f[kMaxN];
  // the FP64 kernel's runtime scalars as float pairs: per direction 1/h, 1/(2h), sigma interior,
  // sigma Dirichlet, a h_e h_f
  float dfs[3][5][2];
  // the plane kernel's per-direction coefficients, each times s = a h_e h_f: h^-1 / 2 and h^-1 (end terms at
  // interior and Dirichlet ends), the interior and Dirichlet penalties, and the cell stiffness s h^-1 K1
  float fint[3], fbnd[3], sint[3], sbnd[3];
  float K1s[3][kMaxN * kMaxN];
  // quadrature points and right-hand sides: the box's first vertex, Gauss points and weights on [0, 1],
  // S[q][i] = l_i(x_q)
  double origin[3], xq[kMaxN], wq[kMaxN], S[kMaxN * kMaxN];
  const int32_t* skip;
};

template <typename Real>
struct DgTab;
template <>
struct DgTab<double> {
  static __device__ __forceinline__ const double* K1(const DgArgs& a) { return a.K1; }
  static __device__ __forceinline__ const double* M1(const DgArgs& a) { return a.M1; }
  static __device__ __forceinline__ const double* d0(const DgArgs& a) { return a.d0; }
  static __device__ __forceinline__ const double* d1(const DgArgs& a) { return a.d1; }
};
template <>
struct DgTab<float> {
  static __device__ __forceinline__ const float* K1(const DgArgs& a) { return a.K1f; }
  static __device__ __forceinline__ const float* M1(const DgArgs& a) { return a.M1f; }
  static __device__ __forceinline__ const float* d0(const DgArgs& a) { return a.d0f; }
  static __device__ __forceinline__ const float* d1(const DgArgs& a) { return a.d1f; }
};

// Line `line` (0 .. n^2 - 1) of an n^3 block along direction dir: first element and stride.
template <int N>
__device__ __forceinline__ void dg_line(int dir, int line, int* base, int* stride) {
  constexpr int N2 = N * N;
  const int p = line % N, q = line / N;
  *base = dir == 0 ? N * p + N2 * q : (dir == 1 ? p + N2 * q : p + N * q);
  *stride = dir == 0 ? 1 : (dir == 1 ? N : N2);
}

// out = M along direction dir on one line (M a compile-time-indexed 1D table)
template <int N, typename Real>
__device__ __forceinline__ void dg_sweep(const Real* in, Real* out, const Real* M, int dir, int line) {
  int base, stride;
  dg_line<N>(dir, line, &base, &stride);
  Real x[N];
#pragma unroll
  for (int i = 0; i < N; ++i) x[i] = in[base + i * stride];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    Real s = Real(0);
#pragma unroll
    for (int j = 0; j < N; ++j) s += M[i * N + j] * x[j];
    out[base + i * stride] = s;
  }
}

// The 1D SIPG operator along direction d on one line of cell `cell` (own data u in shared memory, the
// neighbours' lines read from src), times a h_e h_f.
template <int N, typename Real>
__device__ __forceinline__ void dg_line_sipg(const DgArgs& a, const Real* __restrict__ u, Real* __restrict__ out,
                                             const Real* __restrict__ src, int64_t cell, const int* cidx, int d,
                                             int line) {
  constexpr int N3 = N * N * N, K = N - 1;
  const Real* K1 = DgTab<Real>::K1(a);
  const Real* d0 = DgTab<Real>::d0(a);
  const Real* d1 = DgTab<Real>::d1(a);
  int base, stride;
  dg_line<N>(d, line, &base, &stride);
  const int dims[3] = {a.nx, a.ny, a.nz};
  const Real hinv = Real(a.hinv[d]);
  Real x[N], y[N];
#pragma unroll
  for (int i = 0; i < N; ++i) x[i] = u[base + i * stride];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    Real s = Real(0);
#pragma unroll
    for (int j = 0; j < N; ++j) s += K1[i * N + j] * x[j];
    y[i] = s * hinv;
  }
  const bool lo_nb = cidx[d] > 0, hi_nb = cidx[d] + 1 < dims[d];
  const int64_t step = d == 0 ? 1 : (d == 1 ? (int64_t)a.nx : (int64_t)a.nx * a.ny);
  // at an interior end the own and the neighbour's rank-one terms share the vector d0 (d1): one update
  // with the jump of the end values
  if (lo_nb) {
    const Real* w = src + (cell - step) * N3 + base;
    Real wv[N];
#pragma unroll
    for (int j = 0; j < N; ++j) wv[j] = w[j * stride];
    Real g = Real(0);
#pragma unroll
    for (int j = 0; j < N; ++j) g += d0[j] * x[j] + d1[j] * wv[j];
    const Real jmp = x[0] - wv[K];
    const Real t = Real(0.5) * jmp * hinv;
#pragma unroll
    for (int i = 0; i < N; ++i) y[i] += d0[i] * t;
    y[0] += Real(0.5) * g * hinv + Real(a.sig_int[d]) * jmp;
  } else if ((a.dmask >> (2 * d)) & 1u) {
    Real g = Real(0);
#pragma unroll
    for (int j = 0; j < N; ++j) g += d0[j] * x[j];
    const Real t = x[0] * hinv;
#pragma unroll
    for (int i = 0; i < N; ++i) y[i] += d0[i] * t;
    y[0] += g * hinv + Real(a.sig_bnd[d]) * x[0];
  }
  if (hi_nb) {
    const Real* w = src + (cell + step) * N3 + base;
    Real wv[N];
#pragma unroll
    for (int j = 0; j < N; ++j) wv[j] = w[j * stride];
    Real g = Real(0);
#pragma unroll
    for (int j = 0; j < N; ++j) g += d1[j] * x[j] + d0[j] * wv[j];
    const Real jmp = x[K] - wv[0];
    const Real t = Real(0.5) * jmp * hinv;
#pragma unroll
    for (int i = 0; i < N; ++i) y[i] -= d1[i] * t;
    y[K] += Real(a.sig_int[d]) * jmp - Real(0.5) * g * hinv;
  } else if ((a.dmask >> (2 * d + 1)) & 1u) {
    Real g = Real(0);
#pragma unroll
    for (int j = 0; j < N; ++j) g += d1[j] * x[j];
    const Real t = x[K] * hinv;
#pragma unroll
    for (int i = 0; i < N; ++i) y[i] -= d1[i] * t;
    y[K] += Real(a.sig_bnd[d]) * x[K] - g * hinv;
  }
  const Real sc = Real(a.scale[d]);
#pragma unroll
  for (int i = 0; i < N; ++i) out[base + i * stride] = sc * y[i];
}

template <int N, typename Real>
__global__ void __launch_bounds__(128) dg_vmult_kernel(const __grid_constant__ DgArgs a, const Real* __restrict__ src,
                                                        Real* __restrict__ dst) {
  constexpr int N2 = N * N, N3 = N2 * N;
  constexpr int CB = 128 / N2 > 0 ? 128 / N2 : 1;
  constexpr int CH = CB * N3;  // DoFs of one batch of cells
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* U = reinterpret_cast<Real*>(smem_raw);  // u, then T1
  Real* P = U + CH;                             // P, then M_z (T1 + T2)
  Real* Q = P + CH;                             // Q, then M_y T3
  Real* R = Q + CH;
  Real* T2 = R + CH;
  Real* T3 = T2 + CH;
  const int cl = threadIdx.x / N2;
  const int r = threadIdx.x - cl * N2;
  const bool lane_ok = cl < CB;
  const Real* M1 = DgTab<Real>::M1(a);
  const int64_t total = a.n_cells * N3;
  const int64_t nbatch = (a.n_cells + CB - 1) / CB;
  for (int64_t bt = blockIdx.x; bt < nbatch; bt += gridDim.x) {
    const int64_t first = bt * CB * (int64_t)N3;
    const bool full = first + CH <= total;
    if (full) {
#pragma unroll 4
      for (int i = threadIdx.x; i < CH; i += 128) U[i] = src[first + i];
    } else {
      for (int i = threadIdx.x; i < CH; i += 128) U[i] = first + i < total ? src[first + i] : Real(0);
    }
    __syncthreads();
    const int64_t cell = bt * CB + cl;
    const bool act = lane_ok && cell < a.n_cells;
    const int off = (lane_ok ? cl : 0) * N3;
    if (act) {
      // fewer than 2^31 cells (fewer than 2^31 DoFs): 32-bit coordinates
      const unsigned c32 = (unsigned)cell, q = c32 / (unsigned)a.nx, cz = q / (unsigned)a.ny;
      const int cidx[3] = {(int)(c32 - q * (unsigned)a.nx), (int)(q - cz * (unsigned)a.ny), (int)cz};
      dg_line_sipg<N, Real>(a, U + off, P + off, src, cell, cidx, 0, r);
      dg_line_sipg<N, Real>(a, U + off, Q + off, src, cell, cidx, 1, r);
      dg_line_sipg<N, Real>(a, U + off, R + off, src, cell, cidx, 2, r);
    }
    __syncthreads();
    if (act) {
      dg_sweep<N, Real>(P + off, U + off, M1, 1, r);   // T1 = M_y P
      dg_sweep<N, Real>(Q + off, T2 + off, M1, 0, r);  // T2 = M_x Q
      dg_sweep<N, Real>(R + off, T3 + off, M1, 0, r);  // T3 = M_x R
    }
    __syncthreads();
    if (act) {
      int base, stride;
      dg_line<N>(2, r, &base, &stride);
      Real x[N];
#pragma unroll
      for (int i = 0; i < N; ++i) x[i] = U[off + base + i * stride] + T2[off + base + i * stride];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        Real s = Real(0);
#pragma unroll
        for (int j = 0; j < N; ++j) s += M1[i * N + j] * x[j];
        P[off + base + i * stride] = s;                  // M_z (T1 + T2)
      }
      dg_sweep<N, Real>(T3 + off, Q + off, M1, 1, r);  // M_y T3
    }
    __syncthreads();
    if (full) {
#pragma unroll 4
      for (int i = threadIdx.x; i < CH; i += 128) dst[first + i] = P[i] + Q[i];
    } else {
      for (int i = threadIdx.x; i < CH; i += 128)
        if (first + i < total) dst[first + i] = P[i] + Q[i];
    }
  }
}

// FP32 plane kernel (degrees 1..5).  The same Kronecker sum, ordered so that two of the three
// directions never leave registers:
//   y = M_z C + D,   C = M_y (s_x L_x u) + M_x (s_y L_y u),   D = M_x M_y R,   R = s_z L_z u.
// A CTA takes CB consecutive cells (CB N plane tasks, at most 128 threads).  Three phases per batch:
//   z-lines (one task per line of a cell, several per thread): R from the cell's z-line, with the
//     z-neighbours' z-lines read from global memory (coalesced: a z-line task reads one point per
//     plane), requested before the batch's staging completes;
//   planes (one task per z-plane of a cell): L_x along the plane's rows and L_y along its columns, the
//     x-neighbours' planes taken from the staged chunk (cells c0 - 1 .. c0 + CB) and the y-neighbours'
//     planes from two more staged chunks (cells c0 -/+ nx ..), the masses M_y and M_x applied in
//     registers row by row and column by column; C written over the task's own plane of the y-lower
//     chunk, D over its plane of R;
//   z-lines: y = M_z C + D, stored straight to dst.
// The staged chunks are asynchronous 16-byte copies from a 16-byte aligned start below the chunk,
// indexed from the shift; points outside the vector read as zero (and are never used: the face flags
// of a cell select which neighbour data enter).  The next batch's own and y-upper chunks are requested
// before the last phase of the current one, which reads neither.
// Measured and dropped (p = 4, 65.5M DoFs, against 0.32 ms): two planes per thread as the lanes of packed
// FFMA2 values (half the threads, twice the shared loads each: 0.36-0.43 ms), 21 cells per batch for five
// CTAs per SM (0.36 ms).
template <int N>
struct DgPlane {
  static constexpr int N2 = N * N, N3 = N2 * N;
  static constexpr int CB = 128 / N;  // cells per batch: N z-planes per cell
  static constexpr int region(int len) { return (len + 6 + 3) & ~3; }  // staged length + alignment shift
  static constexpr int UL = region((CB + 2) * N3), YL = region(CB * N3), RL = (CB * N3 + 3) & ~3;
  static constexpr size_t SMEM = (size_t)(UL + 2 * YL + RL) * sizeof(float) + 16 * ((CB + 3) / 4);
};

// Copy src[g0, g0 + len) (zero outside [0, total)) to s' = s + (g0 mod 4) with asynchronous 16-byte copies
// (cp.async; the caller waits with cp.async.wait_all before its barrier) and plain stores for the quads at
// the ends of the vector; returns s + (g0 mod 4), the chunk's first point.  src 16-byte aligned, s 16-byte
// aligned with room for len + 6 floats.
__device__ __forceinline__ float* dg_stage(float* s, const float* __restrict__ src, int64_t g0, int len,
                                           int64_t total) {
  const int64_t a0 = g0 & ~(int64_t)3;
  const int sh = (int)(g0 - a0);
  const int nq = (len + sh + 3) >> 2;
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    const int64_t g = a0 + 4 * (int64_t)q;
    if (g >= 0 && g + 4 <= total) {
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(s + 4 * q)),
                   "l"(src + g)
                   : "memory");
    } else {
      float4 v;
      v.x = (g >= 0 && g < total) ? src[g] : 0.f;
      v.y = (g + 1 >= 0 && g + 1 < total) ? src[g + 1] : 0.f;
      v.z = (g + 2 >= 0 && g + 2 < total) ? src[g + 2] : 0.f;
      v.w = (g + 3 >= 0 && g + 3 < total) ? src[g + 3] : 0.f;
      reinterpret_cast<float4*>(s)[q] = v;
    }
  }
  return s + sh;
}

__device__ __forceinline__ void dg_stage_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// One line x of the 1D SIPG operator of direction D, times the direction's scale s, in registers:
//   y = s h^-1 K1 x + (lower end) d0 tl + e_0 (fl (g0 + gl) + sl jl) - (upper end) d1 th + e_K (sh jh - fh (g1 + gh)),
// jl = x_0 - wl, tl = fl jl, g0 = d0 . x, jh = x_K - wh, th = fh jh, g1 = d1 . x; (fl, sl) are
// (s h^-1 / 2, s sigma_int) at an interior end, (s h^-1, s sigma_Dirichlet) at a Dirichlet end and zero at
// a natural end; (wl, gl) the lower neighbour's value at its upper end and d1 . w (zero without one),
// (wh, gh) the upper neighbour's value at its lower end and d0 . w.  The scale is folded into the
// stiffness table (K1s[D] = s h^-1 K1).
template <int N, int D>
__device__ __forceinline__ void dg_line_reg(const DgArgs& a, const float (&x)[N], float (&y)[N], float fl, float sl,
                                            float wl, float gl, float fh, float shc, float wh, float gh) {
  constexpr int K = N - 1;
  float g0 = a.d0f[0] * x[0], g1 = a.d1f[0] * x[0];
#pragma unroll
  for (int j = 1; j < N; ++j) {
    g0 = fmaf(a.d0f[j], x[j], g0);
    g1 = fmaf(a.d1f[j], x[j], g1);
  }
  const float jl = x[0] - wl, jh = x[K] - wh;
  const float tl = fl * jl, tn = -fh * jh;  // minus the upper end's factor
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float s = fmaf(a.d1f[i], tn, a.d0f[i] * tl);
#pragma unroll
    for (int j = 0; j < N; ++j) s = fmaf(a.K1s[D][i * N + j], x[j], s);
    y[i] = s;
  }
  y[0] = fmaf(fl, g0 + gl, fmaf(sl, jl, y[0]));
  y[K] = fmaf(shc, jh, fmaf(-fh, g1 + gh, y[K]));
}

// A neighbour line's contribution: its value at the shared end and its end derivative sum, or zeros
// without the neighbour (a select, not a product: the staged cell beside a boundary face belongs to
// another row of cells).
template <int N, bool LOWER>
__device__ __forceinline__ void dg_nb_end(const DgArgs& a, const float (&w)[N], bool has, float* wv, float* g) {
  float s = (LOWER ? a.d1f[0] : a.d0f[0]) * w[0];
#pragma unroll
  for (int j = 1; j < N; ++j) s = fmaf(LOWER ? a.d1f[j] : a.d0f[j], w[j], s);
  *g = has ? s : 0.f;
  *wv = has ? (LOWER ? w[N - 1] : w[0]) : 0.f;
}

// End coefficients of direction d for a cell with face flags f (bit 2d: lower neighbour, 2d+1: upper).
__device__ __forceinline__ void dg_end_coefs(const DgArgs& a, int d, int f, float* fl, float* sl, float* fh,
                                             float* shc) {
  const bool lo = (f >> (2 * d)) & 1, hi = (f >> (2 * d + 1)) & 1;
  const bool dlo = (a.dmask >> (2 * d)) & 1u, dhi = (a.dmask >> (2 * d + 1)) & 1u;
  *fl = lo ? a.fint[d] : (dlo ? a.fbnd[d] : 0.f);
  *sl = lo ? a.sint[d] : (dlo ? a.sbnd[d] : 0.f);
  *fh = hi ? a.fint[d] : (dhi ? a.fbnd[d] : 0.f);
  *shc = hi ? a.sint[d] : (dhi ? a.sbnd[d] : 0.f);
}

__device__ __forceinline__ float2 dg_f2(float v) { return make_float2(v, v); }

// dg_line_reg on two lines at once (the lanes of each float2, each with its own end coefficients) with
// packed multiply-adds; fhn is minus the upper end's factor.
template <int N, int D>
__device__ __forceinline__ void dg_line_reg2(const DgArgs& a, const float2 (&x)[N], float2 (&y)[N], float2 fl, float2 sl,
                                             float2 wl, float2 gl, float2 fhn, float2 shc, float2 wh, float2 gh) {
  constexpr int K = N - 1;
  float2 g0 = __fmul2_rn(dg_f2(a.d0f[0]), x[0]);
  float2 g1 = __fmul2_rn(dg_f2(a.d1f[0]), x[0]);
#pragma unroll
  for (int j = 1; j < N; ++j) {
    g0 = __ffma2_rn(dg_f2(a.d0f[j]), x[j], g0);
    g1 = __ffma2_rn(dg_f2(a.d1f[j]), x[j], g1);
  }
  const float2 jl = __ffma2_rn(dg_f2(-1.f), wl, x[0]);
  const float2 jh = __ffma2_rn(dg_f2(-1.f), wh, x[K]);
  const float2 tl = __fmul2_rn(fl, jl);
  const float2 tn = __fmul2_rn(fhn, jh);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float2 s = __ffma2_rn(dg_f2(a.d1f[i]), tn, __fmul2_rn(dg_f2(a.d0f[i]), tl));
#pragma unroll
    for (int j = 0; j < N; ++j) s = __ffma2_rn(dg_f2(a.K1s[D][i * N + j]), x[j], s);
    y[i] = s;
  }
  y[0] = __ffma2_rn(fl, __ffma2_rn(dg_f2(1.f), g0, gl), __ffma2_rn(sl, jl, y[0]));
  y[K] = __ffma2_rn(shc, jh, __ffma2_rn(fhn, __ffma2_rn(dg_f2(1.f), g1, gh), y[K]));
}

// dg_nb_end on two neighbour lines at once, each lane with its own neighbour flag.
template <int N, bool LOWER>
__device__ __forceinline__ void dg_nb_end2(const DgArgs& a, const float2 (&w)[N], bool hx, bool hy, float2* wv,
                                           float2* g) {
  float2 s = __fmul2_rn(dg_f2(LOWER ? a.d1f[0] : a.d0f[0]), w[0]);
#pragma unroll
  for (int j = 1; j < N; ++j) s = __ffma2_rn(dg_f2(LOWER ? a.d1f[j] : a.d0f[j]), w[j], s);
  const float2 v = LOWER ? w[N - 1] : w[0];
  *g = make_float2(hx ? s.x : 0.f, hy ? s.y : 0.f);
  *wv = make_float2(hx ? v.x : 0.f, hy ? v.y : 0.f);
}

// End coefficients of direction d for the two lanes' cells (face flags fx, fy), the upper end's factor negated.
__device__ __forceinline__ void dg_end_coefs2(const DgArgs& a, int d, int fx, int fy, float2* fl, float2* sl,
                                              float2* fhn, float2* shc) {
  float a0, a1, a2, a3, b0, b1, b2, b3;
  dg_end_coefs(a, d, fx, &a0, &a1, &a2, &a3);
  dg_end_coefs(a, d, fy, &b0, &b1, &b2, &b3);
  *fl = make_float2(a0, b0);
  *sl = make_float2(a1, b1);
  *fhn = make_float2(-a2, -b2);
  *shc = make_float2(a3, b3);
}

template <int N>
__global__ void __launch_bounds__(128, N <= 3 ? 6 : (N <= 5 ? 4 : 2))
    dg_vmult_plane_kernel(const __grid_constant__ DgArgs a, const float* __restrict__ src, float* __restrict__ dst) {
  using Sh = DgPlane<N>;
  constexpr int N2 = Sh::N2, N3 = Sh::N3, CB = Sh::CB;
  constexpr int RZ = (CB * N2 + 127) / 128;  // z-line tasks per thread
  constexpr int RP = RZ / 2 > 0 ? RZ / 2 : 1;  // pairs of them (RZ >= 2 at every degree)
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) float dsm[];
  float* const Us = dsm;            // cells c0 - 1 .. c0 + CB
  float* const Yls = Us + Sh::UL;   // cells c0 - nx .., then C over the planes
  float* const Yhs = Yls + Sh::YL;  // cells c0 + nx ..
  float* const Rb = Yhs + Sh::YL;   // R, then D over the planes
  int* const cflag = reinterpret_cast<int*>(Rb + Sh::RL);
  const float* M = a.M1f;
  const int64_t ncell = a.n_cells, total = ncell * N3;
  const int64_t sxy = (int64_t)a.nx * a.ny;
  const int zoff = (int)(sxy * N3);  // fewer than 2^31 DoFs
  const int64_t nbatch = (ncell + CB - 1) / CB;
  // the plane task of this thread: z-plane pk of cell pc of the batch
  const int pc = threadIdx.x / N, pk = threadIdx.x - pc * N;
  const int poff = pc * N3 + N2 * pk;
  // staging of the batch's own chunk (with the x-neighbours) and of its y-upper chunk is issued while the
  // previous batch finishes (its last phase reads neither buffer)
  float* U = nullptr;
  float* Yh = nullptr;
  if (blockIdx.x < nbatch) {
    const int64_t c0 = (int64_t)blockIdx.x * CB;
    U = dg_stage(Us, src, (c0 - 1) * N3, (CB + 2) * N3, total) + N3;  // U: cell c0
    Yh = dg_stage(Yhs, src, (c0 + a.nx) * N3, CB * N3, total);
  }
  for (int64_t bt = blockIdx.x; bt < nbatch; bt += gridDim.x) {
    const int64_t c0 = bt * CB;
    const int nc = (int)std::min<int64_t>(CB, ncell - c0);  // cells in this batch
    if (threadIdx.x < CB) {
      // face flags: bit 2d lower neighbour in direction d, 2d + 1 upper (fewer than 2^31 cells)
      const int64_t cell = c0 + threadIdx.x;
      int f = 0;
      if (cell < ncell) {
        const unsigned c32 = (unsigned)cell, q = c32 / (unsigned)a.nx, cz = q / (unsigned)a.ny;
        const unsigned cx = c32 - q * (unsigned)a.nx, cy = q - cz * (unsigned)a.ny;
        f = (cx > 0) | ((cx + 1 < (unsigned)a.nx) << 1) | ((cy > 0) << 2) | ((cy + 1 < (unsigned)a.ny) << 3) |
            ((cz > 0) << 4) | ((cz + 1 < (unsigned)a.nz) << 5);
      }
      cflag[threadIdx.x] = f;
    }
    float* const Yl = dg_stage(Yls, src, (c0 - a.nx) * N3, CB * N3, total);
    const float* const srcb = src + c0 * N3;
    // the z-neighbours' lines of this thread's z-line tasks, requested before the staging completes (a
    // cell has a z-lower neighbour iff its index is at least nx ny, a z-upper one iff index + nx ny is
    // below the cell count); rounds 2p and 2p + 1 of a thread's tasks are the lanes of float2 values
    float2 wlo[RP][N], whi[RP][N];
    float wlo1[N], whi1[N];
#pragma unroll
    for (int r = 0; r < RZ; ++r) {
      const int t = threadIdx.x + 128 * r;
      const int c = t / N2, o = c * N3 + (t - c * N2);
      const bool lo = c < nc && c0 + c >= sxy, hi = c < nc && c0 + c + sxy < ncell;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const float vl = lo ? __ldg(srcb + (o - zoff + N2 * k)) : 0.f;
        const float vh = hi ? __ldg(srcb + (o + zoff + N2 * k)) : 0.f;
        if (r < 2 * RP) {
          if (r & 1) {
            wlo[r / 2][k].y = vl;
            whi[r / 2][k].y = vh;
          } else {
            wlo[r / 2][k].x = vl;
            whi[r / 2][k].x = vh;
          }
        } else {
          wlo1[k] = vl;
          whi1[k] = vh;
        }
      }
    }
    dg_stage_wait();
    __syncthreads();
    // z-lines: R = s_z L_z u, two tasks at a time in packed arithmetic (the second lane repeats the first,
    // never stored, where its task lies past the batch's last cell)
#pragma unroll
    for (int q = 0; q < RP; ++q) {
      const int tX = threadIdx.x + 256 * q, tY = tX + 128;
      const int cX = tX / N2, oX = cX * N3 + (tX - cX * N2);
      const int cY = tY / N2, oY = cY * N3 + (tY - cY * N2);
      const bool hy = cY < nc;
      if (cX < nc) {
        const int fX = cflag[cX], fY = hy ? cflag[cY] : fX, oYe = hy ? oY : oX;
        float2 x[N], y[N], wl, gl, wh, gh, fl, sl, fhn, shc;
#pragma unroll
        for (int k = 0; k < N; ++k) x[k] = make_float2(U[oX + N2 * k], U[oYe + N2 * k]);
        dg_nb_end2<N, true>(a, wlo[q], true, true, &wl, &gl);  // zeros already without a neighbour
        dg_nb_end2<N, false>(a, whi[q], true, true, &wh, &gh);
        dg_end_coefs2(a, 2, fX, fY, &fl, &sl, &fhn, &shc);
        dg_line_reg2<N, 2>(a, x, y, fl, sl, wl, gl, fhn, shc, wh, gh);
#pragma unroll
        for (int k = 0; k < N; ++k) {
          Rb[oX + N2 * k] = y[k].x;
          if (hy) Rb[oY + N2 * k] = y[k].y;
        }
      }
    }
    if (RZ & 1) {
      const int t = threadIdx.x + 128 * (RZ - 1);
      const int c = t / N2, o = c * N3 + (t - c * N2);
      if (c < nc) {
        const int f = cflag[c];
        float x[N], y[N];
#pragma unroll
        for (int k = 0; k < N; ++k) x[k] = U[o + N2 * k];
        float wl, gl, wh, gh;
        dg_nb_end<N, true>(a, wlo1, true, &wl, &gl);
        dg_nb_end<N, false>(a, whi1, true, &wh, &gh);
        float fl, sl, fh, shc;
        dg_end_coefs(a, 2, f, &fl, &sl, &fh, &shc);
        dg_line_reg<N, 2>(a, x, y, fl, sl, wl, gl, fh, shc, wh, gh);
#pragma unroll
        for (int k = 0; k < N; ++k) Rb[o + N2 * k] = y[k];
      }
    }
    __syncthreads();
    // planes: D = M_x M_y R, C = M_y (s_x L_x u) + M_x (s_y L_y u), one z-plane per thread
    if (threadIdx.x < CB * N && pc < nc) {
      const int f = cflag[pc];
      {
        float* const rp = Rb + poff;
        float t[N][N];  // M_y R, accumulated row by row of R
#pragma unroll
        for (int n = 0; n < N; ++n) {
          float rr[N];
#pragma unroll
          for (int i = 0; i < N; ++i) rr[i] = rp[N * n + i];
#pragma unroll
          for (int j = 0; j < N; ++j)
#pragma unroll
            for (int i = 0; i < N; ++i) t[j][i] = n == 0 ? M[j * N] * rr[i] : fmaf(M[j * N + n], rr[i], t[j][i]);
        }
#pragma unroll
        for (int j = 0; j < N; ++j)
#pragma unroll
          for (int i = 0; i < N; ++i) {
            float s = M[i * N] * t[j][0];
#pragma unroll
            for (int m = 1; m < N; ++m) s = fmaf(M[i * N + m], t[j][m], s);
            rp[N * j + i] = s;
          }
      }
      const float* const up = U + poff;
      float u[N][N], cacc[N][N];
#pragma unroll
      for (int j = 0; j < N; ++j)
#pragma unroll
        for (int i = 0; i < N; ++i) u[j][i] = up[N * j + i];
      {
        // rows: P = s_x L_x u, accumulated into C = M_y P row by row of P; the x-neighbours' planes are the
        // staged cells beside this one (always in the staging buffer, selected by the face flags)
        float fl, sl, fh, shc;
        dg_end_coefs(a, 0, f, &fl, &sl, &fh, &shc);
        const bool xl = f & 1, xh = (f >> 1) & 1;
#pragma unroll
        for (int m = 0; m < N; ++m) {
          float wn[N], p[N], wl, gl, wh, gh;
#pragma unroll
          for (int i = 0; i < N; ++i) wn[i] = up[N * m + i - N3];
          dg_nb_end<N, true>(a, wn, xl, &wl, &gl);
#pragma unroll
          for (int i = 0; i < N; ++i) wn[i] = up[N * m + i + N3];
          dg_nb_end<N, false>(a, wn, xh, &wh, &gh);
          dg_line_reg<N, 0>(a, u[m], p, fl, sl, wl, gl, fh, shc, wh, gh);
#pragma unroll
          for (int j = 0; j < N; ++j)
#pragma unroll
            for (int i = 0; i < N; ++i) cacc[j][i] = m == 0 ? M[j * N] * p[i] : fmaf(M[j * N + m], p[i], cacc[j][i]);
        }
      }
      float* const ylp = Yl + poff;
      {
        // columns: Q = s_y L_y u, accumulated into C += M_x Q column by column of Q
        float fl, sl, fh, shc;
        dg_end_coefs(a, 1, f, &fl, &sl, &fh, &shc);
        const bool yl = (f >> 2) & 1, yh = (f >> 3) & 1;
        const float* const yhp = Yh + poff;
#pragma unroll
        for (int i = 0; i < N; ++i) {
          float x[N], wn[N], q[N], wl, gl, wh, gh;
#pragma unroll
          for (int j = 0; j < N; ++j) x[j] = u[j][i];
#pragma unroll
          for (int j = 0; j < N; ++j) wn[j] = ylp[N * j + i];
          dg_nb_end<N, true>(a, wn, yl, &wl, &gl);
#pragma unroll
          for (int j = 0; j < N; ++j) wn[j] = yhp[N * j + i];
          dg_nb_end<N, false>(a, wn, yh, &wh, &gh);
          dg_line_reg<N, 1>(a, x, q, fl, sl, wl, gl, fh, shc, wh, gh);
#pragma unroll
          for (int j = 0; j < N; ++j)
#pragma unroll
            for (int ii = 0; ii < N; ++ii) cacc[j][ii] = fmaf(M[ii * N + i], q[j], cacc[j][ii]);
        }
      }
      // C over the task's own plane of the y-lower staging (read only by this task, all reads done)
#pragma unroll
      for (int j = 0; j < N; ++j)
#pragma unroll
        for (int i = 0; i < N; ++i) ylp[N * j + i] = cacc[j][i];
    }
    __syncthreads();
    if (bt + gridDim.x < nbatch) {
      const int64_t n0 = (bt + gridDim.x) * CB;
      U = dg_stage(Us, src, (n0 - 1) * N3, (CB + 2) * N3, total) + N3;
      Yh = dg_stage(Yhs, src, (n0 + a.nx) * N3, CB * N3, total);
    }
    // z-lines: y = M_z C + D, two tasks at a time in packed arithmetic
    {
      float* const dstb = dst + c0 * N3;
#pragma unroll
      for (int q = 0; q < RP; ++q) {
        const int tX = threadIdx.x + 256 * q, tY = tX + 128;
        const int cX = tX / N2, oX = cX * N3 + (tX - cX * N2);
        const int cY = tY / N2, oY = cY * N3 + (tY - cY * N2);
        const bool hy = cY < nc;
        if (cX < nc) {
          const int oYe = hy ? oY : oX;
          float2 cc[N], dd[N];
#pragma unroll
          for (int k = 0; k < N; ++k) {
            cc[k] = make_float2(Yl[oX + N2 * k], Yl[oYe + N2 * k]);
            dd[k] = make_float2(Rb[oX + N2 * k], Rb[oYe + N2 * k]);
          }
#pragma unroll
          for (int k = 0; k < N; ++k) {
            float2 s = dd[k];
#pragma unroll
            for (int m = 0; m < N; ++m) s = __ffma2_rn(dg_f2(M[k * N + m]), cc[m], s);
            dstb[oX + N2 * k] = s.x;
            if (hy) dstb[oY + N2 * k] = s.y;
          }
        }
      }
      if (RZ & 1) {
        const int t = threadIdx.x + 128 * (RZ - 1);
        const int c = t / N2, o = c * N3 + (t - c * N2);
        if (c < nc) {
          float cc[N], dd[N];
#pragma unroll
          for (int k = 0; k < N; ++k) {
            cc[k] = Yl[o + N2 * k];
            dd[k] = Rb[o + N2 * k];
          }
#pragma unroll
          for (int k = 0; k < N; ++k) {
            float s = dd[k];
#pragma unroll
            for (int m = 0; m < N; ++m) s = fmaf(M[k * N + m], cc[m], s);
            dstb[o + N2 * k] = s;
          }
        }
      }
    }
    __syncthreads();
  }
}

// FP64 data in double-float arithmetic (the native FP64 kernel runs at the FP64 FMA rate, 1/62 of the
// FP32 rate on GB300): the same phases, with values split into float pairs when loaded and joined back
// to FP64 when stored, the 1D tables split at compile time, and the per-direction scalars split on the
// host.
template <int N, int W>  // W: 0 K1, 1 M1, 2 d0, 3 d1
__device__ __forceinline__ constexpr double dg_tab(int i) {
  return W == 0 ? DgConst<N>::K1(i) : W == 1 ? DgConst<N>::M1(i) : W == 2 ? DgConst<N>::d0(i) : DgConst<N>::d1(i);
}

// y_i = sum_j T[i][j] x_j (T = K1 or M1)
template <int N, int W>
__device__ __forceinline__ void dg_contract_df(const df (&x)[N], df (&y)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float s, t;
    df_prod(x[0], split_hi(dg_tab<N, W>(i * N)), split_lo(dg_tab<N, W>(i * N)), s, t);
#pragma unroll
    for (int j = 1; j < N; ++j) df_prod_acc(x[j], split_hi(dg_tab<N, W>(i * N + j)), split_lo(dg_tab<N, W>(i * N + j)), s, t);
    y[i] = df_fast_norm(s, t);
  }
}

// sum_j v_j x_j + sum_j w_j z_j (v, w = d0 or d1)
template <int N, int V, int W>
__device__ __forceinline__ df dg_dot2_df(const df (&x)[N], const df (&z)[N]) {
  float s, t;
  df_prod(x[0], split_hi(dg_tab<N, V>(0)), split_lo(dg_tab<N, V>(0)), s, t);
#pragma unroll
  for (int j = 1; j < N; ++j) df_prod_acc(x[j], split_hi(dg_tab<N, V>(j)), split_lo(dg_tab<N, V>(j)), s, t);
#pragma unroll
  for (int j = 0; j < N; ++j) df_prod_acc(z[j], split_hi(dg_tab<N, W>(j)), split_lo(dg_tab<N, W>(j)), s, t);
  return df_fast_norm(s, t);
}
template <int N, int V>
__device__ __forceinline__ df dg_dot_df(const df (&x)[N]) {
  float s, t;
  df_prod(x[0], split_hi(dg_tab<N, V>(0)), split_lo(dg_tab<N, V>(0)), s, t);
#pragma unroll
  for (int j = 1; j < N; ++j) df_prod_acc(x[j], split_hi(dg_tab<N, V>(j)), split_lo(dg_tab<N, V>(j)), s, t);
  return df_fast_norm(s, t);
}

// x * c and acc + x * c with c = (ch, cl)
__device__ __forceinline__ df df_mul_c(df x, float ch, float cl) {
  float s, t;
  df_prod(x, ch, cl, s, t);
  return df_fast_norm(s, t);
}
__device__ __forceinline__ df df_fma_c(df x, float ch, float cl, df acc) {
  float s = acc.hi, t = acc.lo;
  df_prod_acc(x, ch, cl, s, t);
  return df_fast_norm(s, t);
}

template <int N>
__device__ __forceinline__ void dg_sweep_df(const df* in, df* out, int dir, int line) {
  int base, stride;
  dg_line<N>(dir, line, &base, &stride);
  df x[N], y[N];
#pragma unroll
  for (int i = 0; i < N; ++i) x[i] = in[base + i * stride];
  dg_contract_df<N, 1>(x, y);
#pragma unroll
  for (int i = 0; i < N; ++i) out[base + i * stride] = y[i];
}

template <int N>
__device__ __forceinline__ void dg_line_sipg_df(const DgArgs& a, const df* __restrict__ u, df* __restrict__ out,
                                                const double* __restrict__ src, int64_t cell, const int* cidx,
                                                int d, int line) {
  constexpr int N3 = N * N * N, K = N - 1;
  int base, stride;
  dg_line<N>(d, line, &base, &stride);
  const int dims[3] = {a.nx, a.ny, a.nz};
  const float(*c)[2] = a.dfs[d];  // 0: 1/h, 1: 1/(2h), 2: sigma interior, 3: sigma Dirichlet, 4: scale
  df x[N], y[N];
#pragma unroll
  for (int i = 0; i < N; ++i) x[i] = u[base + i * stride];
  dg_contract_df<N, 0>(x, y);
#pragma unroll
  for (int i = 0; i < N; ++i) y[i] = df_mul_c(y[i], c[0][0], c[0][1]);
  const bool lo_nb = cidx[d] > 0, hi_nb = cidx[d] + 1 < dims[d];
  const int64_t step = d == 0 ? 1 : (d == 1 ? (int64_t)a.nx : (int64_t)a.nx * a.ny);
  if (lo_nb) {
    df wv[N];
#pragma unroll
    for (int j = 0; j < N; ++j) wv[j] = df_split(src[(cell - step) * N3 + base + j * stride]);
    const df g = dg_dot2_df<N, 2, 3>(x, wv);
    const df jmp = df_add(x[0], df_neg(wv[K]));
    const df t = df_mul_c(jmp, c[1][0], c[1][1]);
#pragma unroll
    for (int i = 0; i < N; ++i) y[i] = df_fma_c(t, split_hi(dg_tab<N, 2>(i)), split_lo(dg_tab<N, 2>(i)), y[i]);
    y[0] = df_fma_c(jmp, c[2][0], c[2][1], df_fma_c(g, c[1][0], c[1][1], y[0]));
  } else if ((a.dmask >> (2 * d)) & 1u) {
    const df g = dg_dot_df<N, 2>(x);
    const df t = df_mul_c(x[0], c[0][0], c[0][1]);
#pragma unroll
    for (int i = 0; i < N; ++i) y[i] = df_fma_c(t, split_hi(dg_tab<N, 2>(i)), split_lo(dg_tab<N, 2>(i)), y[i]);
    y[0] = df_fma_c(x[0], c[3][0], c[3][1], df_fma_c(g, c[0][0], c[0][1], y[0]));
  }
  if (hi_nb) {
    df wv[N];
#pragma unroll
    for (int j = 0; j < N; ++j) wv[j] = df_split(src[(cell + step) * N3 + base + j * stride]);
    const df g = dg_dot2_df<N, 3, 2>(x, wv);
    const df jmp = df_add(x[K], df_neg(wv[0]));
    const df t = df_neg(df_mul_c(jmp, c[1][0], c[1][1]));
#pragma unroll
    for (int i = 0; i < N; ++i) y[i] = df_fma_c(t, split_hi(dg_tab<N, 3>(i)), split_lo(dg_tab<N, 3>(i)), y[i]);
    y[K] = df_fma_c(jmp, c[2][0], c[2][1], df_fma_c(df_neg(g), c[1][0], c[1][1], y[K]));
  } else if ((a.dmask >> (2 * d + 1)) & 1u) {
    const df g = dg_dot_df<N, 3>(x);
    const df t = df_neg(df_mul_c(x[K], c[0][0], c[0][1]));
#pragma unroll
    for (int i = 0; i < N; ++i) y[i] = df_fma_c(t, split_hi(dg_tab<N, 3>(i)), split_lo(dg_tab<N, 3>(i)), y[i]);
    y[K] = df_fma_c(x[K], c[3][0], c[3][1], df_fma_c(df_neg(g), c[0][0], c[0][1], y[K]));
  }
#pragma unroll
  for (int i = 0; i < N; ++i) out[base + i * stride] = df_mul_c(y[i], c[4][0], c[4][1]);
}

template <int N>
__global__ void __launch_bounds__(128) dg_vmult_df_kernel(const __grid_constant__ DgArgs a,
                                                           const double* __restrict__ src, double* __restrict__ dst) {
  constexpr int N2 = N * N, N3 = N2 * N;
  constexpr int CB = 128 / N2 > 0 ? 128 / N2 : 1;
  constexpr int CH = CB * N3;
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  df* U = reinterpret_cast<df*>(smem_raw);
  df* P = U + CH;
  df* Q = P + CH;
  df* R = Q + CH;
  df* T2 = R + CH;
  df* T3 = T2 + CH;
  const int cl = threadIdx.x / N2;
  const int r = threadIdx.x - cl * N2;
  const bool lane_ok = cl < CB;
  const int64_t total = a.n_cells * N3;
  const int64_t nbatch = (a.n_cells + CB - 1) / CB;
  for (int64_t bt = blockIdx.x; bt < nbatch; bt += gridDim.x) {
    const int64_t first = bt * CB * (int64_t)N3;
    for (int i = threadIdx.x; i < CH; i += 128) U[i] = df_split(first + i < total ? src[first + i] : 0.0);
    __syncthreads();
    const int64_t cell = bt * CB + cl;
    const bool act = lane_ok && cell < a.n_cells;
    const int off = (lane_ok ? cl : 0) * N3;
    if (act) {
      const unsigned c32 = (unsigned)cell, q = c32 / (unsigned)a.nx, cz = q / (unsigned)a.ny;
      const int cidx[3] = {(int)(c32 - q * (unsigned)a.nx), (int)(q - cz * (unsigned)a.ny), (int)cz};
      dg_line_sipg_df<N>(a, U + off, P + off, src, cell, cidx, 0, r);
      dg_line_sipg_df<N>(a, U + off, Q + off, src, cell, cidx, 1, r);
      dg_line_sipg_df<N>(a, U + off, R + off, src, cell, cidx, 2, r);
    }
    __syncthreads();
    if (act) {
      dg_sweep_df<N>(P + off, U + off, 1, r);
      dg_sweep_df<N>(Q + off, T2 + off, 0, r);
      dg_sweep_df<N>(R + off, T3 + off, 0, r);
    }
    __syncthreads();
    if (act) {
      int base, stride;
      dg_line<N>(2, r, &base, &stride);
      df x[N], y[N];
#pragma unroll
      for (int i = 0; i < N; ++i) x[i] = df_add(U[off + base + i * stride], T2[off + base + i * stride]);
      dg_contract_df<N, 1>(x, y);
#pragma unroll
      for (int i = 0; i < N; ++i) P[off + base + i * stride] = y[i];
      dg_sweep_df<N>(T3 + off, Q + off, 1, r);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < CH; i += 128)
      if (first + i < total) dst[first + i] = df_join(df_add(P[i], Q[i]));
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

// Physical quadrature points: x = origin + (cell index + x_q) h per direction, [cell][q][3].
__global__ void dg_qpoints_kernel(const __grid_constant__ DgArgs a, int n, double* __restrict__ out) {
  const int n3 = n * n * n;
  const int64_t total = a.n_cells * n3;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = idx / n3;
    const int q = (int)(idx - cell * n3);
    const int qq[3] = {q % n, (q / n) % n, q / (n * n)};
    const int64_t c[3] = {cell % a.nx, (cell / a.nx) % a.ny, cell / ((int64_t)a.nx * a.ny)};
    for (int d = 0; d < 3; ++d) out[3 * idx + d] = a.origin[d] + ((double)c[d] + a.xq[qq[d]]) * a.h[d];
  }
}

// Load vector of f given at the quadrature points: b_i = sum_q w_q |K| f(x_q) phi_i(x_q), each DoF in its
// own cell (no accumulation across cells).
__global__ void dg_rhs_kernel(const __grid_constant__ DgArgs a, int n, const double* __restrict__ fq,
                              double* __restrict__ b) {
  const int n3 = n * n * n;
  const int64_t total = a.n_cells * n3;
  const double vol = a.h[0] * a.h[1] * a.h[2];
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = idx / n3;
    const int i = (int)(idx - cell * n3);
    const int i1 = i % n, i2 = (i / n) % n, i3 = i / (n * n);
    double s = 0.0;
    for (int q = 0; q < n3; ++q) {
      const int q1 = q % n, q2 = (q / n) % n, q3 = q / (n * n);
      const double w = a.wq[q1] * a.wq[q2] * a.wq[q3];
      s += w * a.S[q1 * n + i1] * a.S[q2 * n + i2] * a.S[q3 * n + i3] * fq[cell * n3 + q];
    }
    b[idx] = s * vol;
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
    a.hinv[d] = 1.0 / op->dg_h[d];
    a.sig_int[d] = op->dg_penalty * n * n / op->dg_h[d];
    a.sig_bnd[d] = op->dg_penalty * n * n * 2.0 / op->dg_h[d];
  }
  a.scale[0] = op->dg_coef * op->dg_h[1] * op->dg_h[2];
  a.scale[1] = op->dg_coef * op->dg_h[0] * op->dg_h[2];
  a.scale[2] = op->dg_coef * op->dg_h[0] * op->dg_h[1];
  a.coef = op->dg_coef;
  a.dmask = op->dirichlet;
  for (int d = 0; d < 3; ++d) {
    a.fint[d] = (float)(0.5 * a.hinv[d] * a.scale[d]);
    a.fbnd[d] = (float)(a.hinv[d] * a.scale[d]);
    a.sint[d] = (float)(a.sig_int[d] * a.scale[d]);
    a.sbnd[d] = (float)(a.sig_bnd[d] * a.scale[d]);
  }
  for (int d = 0; d < 3; ++d) {
    const double v[5] = {a.hinv[d], 0.5 * a.hinv[d], a.sig_int[d], a.sig_bnd[d], a.scale[d]};
    for (int e = 0; e < 5; ++e) {
      a.dfs[d][e][0] = (float)v[e];
      a.dfs[d][e][1] = (float)(v[e] - (double)(float)v[e]);
    }
  }
  const BasisTables& b = op->basis;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double k1 = 0.0, m1 = 0.0;
      for (int q = 0; q < n; ++q) {
        k1 += b.wq[q] * b.Sd[q * n + i] * b.Sd[q * n + j];
        m1 += b.wq[q] * b.S[q * n + i] * b.S[q * n + j];
      }
      a.K1[i * n + j] = k1;
      a.M1[i * n + j] = m1;
      a.K1f[i * n + j] = (float)k1;
      a.M1f[i * n + j] = (float)m1;
    }
  for (int d = 0; d < 3; ++d)
    for (int i = 0; i < n * n; ++i) a.K1s[d][i] = (float)(a.K1[i] * a.hinv[d] * a.scale[d]);
  for (int i = 0; i < n; ++i) {
    a.d0[i] = lagrange_derivative(n, b.gll, i, 0.0);
    a.d1[i] = lagrange_derivative(n, b.gll, i, 1.0);
    a.d0f[i] = (float)a.d0[i];
    a.d1f[i] = (float)a.d1[i];
  }
  for (int d = 0; d < 3; ++d) a.origin[d] = op->dg_origin[d];
  for (int q = 0; q < n; ++q) {
    a.xq[q] = b.xq[q];
    a.wq[q] = b.wq[q];
  }
  for (int i = 0; i < n * n; ++i) a.S[i] = b.S[i];
  a.skip = skip;
  return a;
}

template <int N, typename Real>
static mfx_status run_dg(const mfx_op* op, const Real* src, Real* dst, cudaStream_t s, const int32_t* skip) {
  constexpr int N2 = N * N, N3 = N2 * N;
  constexpr int CB = 128 / N2 > 0 ? 128 / N2 : 1;
  const size_t smem = (size_t)6 * CB * N3 * sizeof(Real);
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

template <int N>
static mfx_status run_dg_plane(const mfx_op* op, const float* src, float* dst, cudaStream_t s, const int32_t* skip) {
  using Sh = DgPlane<N>;
  auto kern = dg_vmult_plane_kernel<N>;
  static int blocks_per_sm = -1;
  if (blocks_per_sm < 0) {
    MFX_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM));
    int b = 0;
    MFX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 128, Sh::SMEM));
    blocks_per_sm = b > 0 ? b : 1;
  }
  const DgArgs a = dg_args(op, skip);
  const int64_t nbatch = (op->n_cells + Sh::CB - 1) / Sh::CB;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(nbatch, (int64_t)device_sm_count() * blocks_per_sm));
  kern<<<grid, 128, Sh::SMEM, s>>>(a, src, dst);
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

template <int N>
static mfx_status run_dg_df(const mfx_op* op, const double* src, double* dst, cudaStream_t s, const int32_t* skip) {
  constexpr int N2 = N * N, N3 = N2 * N;
  constexpr int CB = 128 / N2 > 0 ? 128 / N2 : 1;
  const size_t smem = (size_t)6 * CB * N3 * sizeof(df);
  auto kern = dg_vmult_df_kernel<N>;
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
  // FP32 at degrees 1..5 with a 16-byte aligned source: the plane kernel (its staging loads are 16 bytes
  // wide); otherwise the line kernel
  if (sizeof(Real) == 4 && ((uintptr_t)src & 15) == 0) {
    const float* x = (const float*)src;
    float* y = (float*)dst;
    switch (op->n) {
      case 2: return run_dg_plane<2>(op, x, y, s, skip);
      case 3: return run_dg_plane<3>(op, x, y, s, skip);
      case 4: return run_dg_plane<4>(op, x, y, s, skip);
      case 5: return run_dg_plane<5>(op, x, y, s, skip);
      case 6: return run_dg_plane<6>(op, x, y, s, skip);
      default: break;
    }
  }
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
  if (prec == MFX_F64) {
    const double* x = (const double*)src;
    double* y = (double*)dst;
    switch (op->n) {
      case 2: return run_dg_df<2>(op, x, y, s, skip);
      case 3: return run_dg_df<3>(op, x, y, s, skip);
      case 4: return run_dg_df<4>(op, x, y, s, skip);
      case 5: return run_dg_df<5>(op, x, y, s, skip);
      case 6: return run_dg_df<6>(op, x, y, s, skip);
      case 7: return run_dg_df<7>(op, x, y, s, skip);
      case 8: return run_dg_df<8>(op, x, y, s, skip);
      case 9: return run_dg_df<9>(op, x, y, s, skip);
      default: return set_error(MFX_EUNSUPPORTED, "degree out of range");
    }
  }
  return dg_dispatch<float>(op, (const float*)src, (float*)dst, s, skip);
}

mfx_status launch_dg_qpoints(const mfx_op* op, double* xq, cudaStream_t s) {
  const DgArgs a = dg_args(op, nullptr);
  const int64_t total = op->n_dofs;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)device_sm_count() * 16));
  dg_qpoints_kernel<<<grid, 256, 0, s>>>(a, op->n, xq);
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

mfx_status launch_dg_rhs(const mfx_op* op, const double* fq, double* b, cudaStream_t s) {
  const DgArgs a = dg_args(op, nullptr);
  const int64_t total = op->n_dofs;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)device_sm_count() * 16));
  dg_rhs_kernel<<<grid, 256, 0, s>>>(a, op->n, fq, b);
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
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
