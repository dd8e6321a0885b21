// FP64 structured vmult in double-float arithmetic: the matrix-free operator application of Sec. 3.6
// with the sum factorisation of Sec. 3.1 (values and gradients at the Gauss points by 1D contractions,
// the metric of the Q1 map per quadrature point, Sec. 3.4), on a structured box.
//
// GB300 runs FP64 FMAs at 1/62 of the FP32 rate, so the FP64 operator keeps its vectors and the
// metric in FP64 in HBM but does the arithmetic on pairs of floats (hi + lo, about 48 significant
// bits): every product of a value with a matrix entry is formed exactly by an FMA-based
// error-free transformation, sums are accumulated with two-sum, and the pair is renormalised at
// the end of each contraction.  Values are split into pairs when they are loaded (the 1D
// matrices at compile time) and joined back to FP64 before they are added to dst.  All
// arithmetic uses the round-to-nearest intrinsics, which the compiler never fuses, so the
// error-free transformations stay exact.  The phases are those of the FP32 brick-row kernel
// (vmult_brick_tma2.cuh), with the tile rows moved by 8-byte cp.async copies and the output tile
// added to dst with coalesced FP64 atomics; Dirichlet rows get dst = src inside the kernel.
#pragma once

#include "df.cuh"
#include "vmult_brick.cuh"

namespace mfx {

template <int N, int MAT>
__device__ __forceinline__ void contract_df(const df (&in)[N], df (&out)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float s, t;
    constexpr int dummy = 0;
    (void)dummy;
    df_prod(in[0], split_hi(basis_entry<N, MAT>(i * N)), split_lo(basis_entry<N, MAT>(i * N)), s, t);
#pragma unroll
    for (int j = 1; j < N; ++j)
      df_prod_acc(in[j], split_hi(basis_entry<N, MAT>(i * N + j)), split_lo(basis_entry<N, MAT>(i * N + j)), s, t);
    out[i] = df_fast_norm(s, t);
  }
}

template <int N, int MAT>
__device__ __forceinline__ void contract_t_df(const df (&in)[N], df (&out)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float s, t;
    df_prod(in[0], split_hi(basis_entry<N, MAT>(i)), split_lo(basis_entry<N, MAT>(i)), s, t);
#pragma unroll
    for (int j = 1; j < N; ++j)
      df_prod_acc(in[j], split_hi(basis_entry<N, MAT>(j * N + i)), split_lo(basis_entry<N, MAT>(j * N + i)), s, t);
    out[i] = df_fast_norm(s, t);
  }
}


// Entry (q, j) of M (T = false) or of M^T (T = true).
template <int N, int MAT, bool T>
__device__ __forceinline__ constexpr double mat_entry(int q, int j) {
  return T ? basis_entry<N, MAT>(j * N + q) : basis_entry<N, MAT>(q * N + j);
}

// out = M in (T = false) or M^T in (T = true) in even-odd form.  S and D are reflection symmetric,
// M[n-1-q][n-1-j] = sigma M[q][j] with sigma = +1 for S (symmetric Gauss and Gauss-Lobatto points)
// and -1 for D (the derivative changes sign), and so is M^T.  With e_j = in_j + in_{n-1-j} and
// o_j = in_j - in_{n-1-j} (j < n/2), the half sums A_q = (out_q + sigma out_{n-1-q}) / 2 and
// B_q = (out_q - sigma out_{n-1-q}) / 2 are contractions of half length with the coefficients
// (M[q][j] +- M[q][n-1-j]) / 2 (plus the middle column for odd n in A), and
// out_q = A_q + B_q, out_{n-1-q} = sigma (A_q - B_q); the middle row of odd n is a half-length
// contraction of e (sigma = +1) or o (sigma = -1).  About a quarter fewer double-float operations
// than the direct form at n = 5.
template <int N, int MAT, bool T>
__device__ __forceinline__ void contract_df_eo(const df (&in)[N], df (&out)[N]) {
  constexpr int H = N / 2;
  constexpr bool ODD = (N % 2) == 1;
  constexpr bool SYM = MAT == MAT_S;
  df e[H > 0 ? H : 1], o[H > 0 ? H : 1];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    e[j] = df_add(in[j], in[N - 1 - j]);
    o[j] = df_add(in[j], df_neg(in[N - 1 - j]));
  }
#pragma unroll
  for (int q = 0; q < H; ++q) {
    float s, t;
    df A, B;
    {
      constexpr int j0 = 0;
      const double c0 = 0.5 * (mat_entry<N, MAT, T>(q, j0) + mat_entry<N, MAT, T>(q, N - 1 - j0));
      df_prod(e[0], split_hi(c0), split_lo(c0), s, t);
#pragma unroll
      for (int j = 1; j < H; ++j) {
        const double c = 0.5 * (mat_entry<N, MAT, T>(q, j) + mat_entry<N, MAT, T>(q, N - 1 - j));
        df_prod_acc(e[j], split_hi(c), split_lo(c), s, t);
      }
      if constexpr (ODD) {
        const double c = mat_entry<N, MAT, T>(q, H);
        df_prod_acc(in[H], split_hi(c), split_lo(c), s, t);
      }
      A = df_fast_norm(s, t);
    }
    {
      const double c0 = 0.5 * (mat_entry<N, MAT, T>(q, 0) - mat_entry<N, MAT, T>(q, N - 1));
      df_prod(o[0], split_hi(c0), split_lo(c0), s, t);
#pragma unroll
      for (int j = 1; j < H; ++j) {
        const double c = 0.5 * (mat_entry<N, MAT, T>(q, j) - mat_entry<N, MAT, T>(q, N - 1 - j));
        df_prod_acc(o[j], split_hi(c), split_lo(c), s, t);
      }
      B = df_fast_norm(s, t);
    }
    out[q] = df_add(A, B);
    out[N - 1 - q] = SYM ? df_add(A, df_neg(B)) : df_add(B, df_neg(A));
  }
  if constexpr (ODD) {
    float s, t;
    if constexpr (SYM) {
      const double cm = mat_entry<N, MAT, T>(H, H);
      df_prod(in[H], split_hi(cm), split_lo(cm), s, t);
#pragma unroll
      for (int j = 0; j < H; ++j) {
        const double c = mat_entry<N, MAT, T>(H, j);
        df_prod_acc(e[j], split_hi(c), split_lo(c), s, t);
      }
    } else {
      const double c0 = mat_entry<N, MAT, T>(H, 0);
      df_prod(o[0], split_hi(c0), split_lo(c0), s, t);
#pragma unroll
      for (int j = 1; j < H; ++j) {
        const double c = mat_entry<N, MAT, T>(H, j);
        df_prod_acc(o[j], split_hi(c), split_lo(c), s, t);
      }
    }
    out[H] = df_fast_norm(s, t);
  }
}

template <int N, int CB>
__global__ void __launch_bounds__(BrickShape<N, CB, double>::THREADS, 1)
    brick_vmult_df_kernel(const __grid_constant__ BrickArgs<N, double> a, const double* __restrict__ src,
                          double* __restrict__ dst) {
  using Real = double;
  using Sh = BrickShape<N, CB, Real>;
  constexpr int K = Sh::K, NP = Sh::NP, P2 = Sh::P2, CELL = Sh::CELL, N3 = N * N * N;
  constexpr int PITCH = Sh::PITCH, SKEW = Sh::SKEW, WMAX = Sh::WMAX;
  constexpr bool PREFETCH = false;
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* tiles = reinterpret_cast<Real*>(smem_raw);
  df* A = reinterpret_cast<df*>(tiles + Sh::NBUF * Sh::TILE);
  df* B = A + Sh::CUBES;
  df* C = B + Sh::CUBES;

  const int t = threadIdx.x;
  const int c = t % CB;
  const int r = t / CB;
  const int f = r % N, s = r / N;
  const bool line_ok = t < Sh::LINES;
  // line bases in the cubes
  const int xa2 = Sh::XSWAP ? s : f, xa3 = Sh::XSWAP ? f : s;
  const int xbase = c * CELL + xa3 * P2 + xa2 * NP;  // x-line (a2, a3), stride 1
  const int ybase = c * CELL + s * P2 + f;          // y-line (a1 = f, a3 = s), stride NP
  const int zbase = c * CELL + s * NP + f;          // z-line (a1 = f, a2 = s), stride P2
  // z-line (a1 = f, a2 = s) in the tile: point x = c K + f of rows a3 N + s
  const int zx = c * K + f;
  const int ztile = s * PITCH + zx + (zx / K) * SKEW;  // + a3 * N * PITCH
  const int n_batches = (int)a.n_batches;

  // issue the asynchronous copies of batch bb into tile buffer `buf` (Dirichlet points set to 0);
  // warp w copies tile rows w, w + NWARPS, ...; lanes walk the points of the row
  constexpr int NWARPS = Sh::THREADS / 32, XITERS = (WMAX + 31) / 32;
  const int warp = t >> 5, lane = t & 31;
  auto load_tile = [&](int bb, Real* buf) {
    const BatchInfo bi = batch_info<CB, K>(a, bb);
    for (int row = warp; row < N * N; row += NWARPS) {
      const int a2 = row % N, a3 = row / N;
      const int rflags = (a2 == 0 ? 1 : 0) | (a2 == K ? 2 : 0) | (a3 == 0 ? 4 : 0) | (a3 == K ? 8 : 0);
      const bool rbnd = (rflags & bi.eflags) != 0;
      const Real* g = src + bi.gbase + a.Mx * (a2 + a.My * a3);
      Real* p = buf + row * PITCH;
#pragma unroll
      for (int j = 0; j < XITERS; ++j) {
        const int x = lane + 32 * j;
        if (x < bi.Wm) {
          const bool bnd = rbnd || (x == 0 && bi.xlo) || (x == bi.Wm - 1 && bi.xhi);
          Real* q = p + x + (x / K) * SKEW;
          if (bnd)
            *q = Real(0);
          else
            cp_async(q, g + x);
        }
      }
    }
    cp_async_commit();
  };

  int buf = 0;
  if (Sh::NBUF == 2 && (int)blockIdx.x < n_batches) load_tile(blockIdx.x, tiles);

  for (int b = blockIdx.x; b < n_batches; b += gridDim.x) {
    const BatchInfo bi = batch_info<CB, K>(a, b);
    const int m = bi.m;
    const bool act = line_ok && c < m;
    const Real* Gb = a.metric + (int64_t)b * (6 * N3 * CB) + (xa2 * N + xa3 * N * N) * CB + c;
    Real* T = tiles + buf * Sh::TILE;

    if constexpr (Sh::NBUF == 2) {
      // copies of the next batch go into the other buffer; this batch's copies were issued earlier
      if (b + (int)gridDim.x < n_batches) load_tile(b + gridDim.x, tiles + (buf ^ 1) * Sh::TILE);
      else cp_async_commit();
      cp_async_wait<1>();
    } else {
      load_tile(b, T);
      cp_async_wait<0>();
    }
    // the next batch's metric (float pairs, contiguous per batch) into L2 by the TMA engine, so the
    // metric reads of that batch wait on L2 rather than HBM (k <= 4: Q2 / Q3 / Q4 +3 / +2 / +1 %;
    // at k = 8, 280 KB per batch, it measured 18 % slower)
    if (N <= 5 && warp == 0 && b + (int)gridDim.x < n_batches) {
      constexpr unsigned BYTES = 6u * N3 * CB * 8u, CHUNK = 16384u;
      const char* gn = reinterpret_cast<const char*>(a.metric + (int64_t)(b + gridDim.x) * (6 * N3 * CB));
      for (unsigned off = (unsigned)lane * CHUNK; off < BYTES; off += 32u * CHUNK)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(gn + off),
                     "r"(BYTES - off < CHUNK ? BYTES - off : CHUNK) : "memory");
    }
    // metric of this thread's x-line, consumed four phases later
    Real G[PREFETCH ? 6 : 1][N];
    if (PREFETCH && act) {
#pragma unroll
      for (int e = 0; e < 6; ++e)
#pragma unroll
        for (int q = 0; q < N; ++q) G[e][q] = __ldg(Gb + (e * N3 + q) * CB);
    }
    __syncthreads();
    // 1) S along z: z-lines from the tile into cube A
    if (act) {
      df v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = df_split(T[ztile + j * N * PITCH]);
      contract_df_eo<N, MAT_S, false>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[zbase + j * P2] = o[j];
    }
    __syncthreads();
    // 2) S along y
    if (act) {
      df v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[ybase + j * NP];
      contract_df_eo<N, MAT_S, false>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[ybase + j * NP] = o[j];
    }
    __syncthreads();
    // 3) S along x -> values at Gauss points; D along x kept in registers
    df g1[N];
    if (act) {
      df v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[xbase + j];
      contract_df_eo<N, MAT_S, false>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[xbase + j] = o[j];
      contract_df_eo<N, MAT_D, false>(o, g1);
    }
    __syncthreads();
    // 4) D along y -> B, D along z -> C
    if (act) {
      df v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[ybase + j * NP];
      contract_df_eo<N, MAT_D, false>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) B[ybase + j * NP] = o[j];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[zbase + j * P2];
      contract_df_eo<N, MAT_D, false>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) C[zbase + j * P2] = o[j];
    }
    __syncthreads();
    // 5) quadrature-point metric on the x-line; D_x^T in registers
    df t1[N];
    if (act) {
      df h1[N];
#pragma unroll
      for (int q = 0; q < N; ++q) {
        // the metric is stored as float pairs (hi, lo) in place of the FP64 values
        const float2* Gp = reinterpret_cast<const float2*>(Gb);
        const float2 g00 = __ldg(Gp + (0 * N3 + q) * CB), g01 = __ldg(Gp + (1 * N3 + q) * CB);
        const float2 g02 = __ldg(Gp + (2 * N3 + q) * CB), g11 = __ldg(Gp + (3 * N3 + q) * CB);
        const float2 g12 = __ldg(Gp + (4 * N3 + q) * CB), g22 = __ldg(Gp + (5 * N3 + q) * CB);
        const df G00{g00.x, g00.y}, G01{g01.x, g01.y}, G02{g02.x, g02.y};
        const df G11{g11.x, g11.y}, G12{g12.x, g12.y}, G22{g22.x, g22.y};
        const df u1 = g1[q], u2 = B[xbase + q], u3 = C[xbase + q];
        h1[q] = df_dot3(G00, u1, G01, u2, G02, u3);
        B[xbase + q] = df_dot3(G01, u1, G11, u2, G12, u3);
        C[xbase + q] = df_dot3(G02, u1, G12, u2, G22, u3);
      }
      contract_df_eo<N, MAT_D, true>(h1, t1);
    }
    __syncthreads();
    // 6) D_y^T on B, D_z^T on C
    if (act) {
      df v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = B[ybase + j * NP];
      contract_df_eo<N, MAT_D, true>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) B[ybase + j * NP] = o[j];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = C[zbase + j * P2];
      contract_df_eo<N, MAT_D, true>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) C[zbase + j * P2] = o[j];
    }
    __syncthreads();
    // 7) sum of the three components, S_x^T -> A
    if (act) {
      df v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = df_add3(t1[j], B[xbase + j], C[xbase + j]);
      contract_df_eo<N, MAT_S, true>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[xbase + j] = o[j];
    }
    __syncthreads();
    // 8) S_y^T
    if (act) {
      df v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[ybase + j * NP];
      contract_df_eo<N, MAT_S, true>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[ybase + j * NP] = o[j];
    }
    __syncthreads();
    // 9) S_z^T into the output tile (aliases this batch's input tile, consumed in step 1):
    //    nodes with a1 < K first, then the a1 = K nodes add to the next cell's a1 = 0 node
    df o9[N];
    if (act) {
      df v[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[zbase + j * P2];
      contract_df_eo<N, MAT_S, true>(v, o9);
      if (f < K) {
#pragma unroll
        for (int j = 0; j < N; ++j) T[ztile + j * N * PITCH] = df_join(o9[j]);
      }
    }
    __syncthreads();
    if (act && f == K) {
      if (c < m - 1) {
#pragma unroll
        for (int j = 0; j < N; ++j) T[ztile + j * N * PITCH] += df_join(o9[j]);
      } else {
#pragma unroll
        for (int j = 0; j < N; ++j) T[ztile + j * N * PITCH] = df_join(o9[j]);
      }
    }
    __syncthreads();
    // 10) scatter: coalesced atomic adds, warp per tile row; constrained rows copy src
    for (int row = warp; row < N * N; row += NWARPS) {
      const int a2 = row % N, a3 = row / N;
      const int rflags = (a2 == 0 ? 1 : 0) | (a2 == K ? 2 : 0) | (a3 == 0 ? 4 : 0) | (a3 == K ? 8 : 0);
      const bool rbnd = (rflags & bi.eflags) != 0;
      const int g = bi.gbase + a.Mx * (a2 + a.My * a3);
      const Real* p = T + row * PITCH;
#pragma unroll
      for (int j = 0; j < XITERS; ++j) {
        const int x = lane + 32 * j;
        if (x < bi.Wm) {
          const bool bnd = rbnd || (x == 0 && bi.xlo) || (x == bi.Wm - 1 && bi.xhi);
          if (bnd)
            dst[g + x] = __ldg(src + g + x);
          else
            red_add(dst + g + x, p[x + (x / K) * SKEW]);
        }
      }
    }
    __syncthreads();
    buf ^= (Sh::NBUF - 1);
  }
  if constexpr (Sh::NBUF == 2) cp_async_wait<0>();
}

}  // namespace mfx
