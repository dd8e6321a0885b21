// FP32 brick-row vmult in five synchronised phases (the cell loop of the matrix-free operator,
// Sec. 3.6, with the tensor-product evaluation of Sec. 3.1 on pairs of cells).
//
// The reference gradient at the Gauss points is taken with the derivative of the nodal basis at
// the Gauss points, Sd[q][j] = l_j'(xi_q), next to the values S[q][j] = l_j(xi_q):
//   d/dx u = Sd_x S_y S_z u,  d/dy u = S_x Sd_y S_z u,  d/dz u = S_x S_y Sd_z u,
// so every line of a direction is read from shared memory once and both of its contractions come
// from the same registers.  Per batch of CB cells of one row (lattice rows in shared memory by TMA,
// as in the ten-phase kernel of vmult_brick_tma2.cuh):
//   1) z-lines of the input tile:  A = S_z u,  C = Sd_z u
//   2) y-lines:  A <- S_y A,  B = Sd_y A,  C <- S_y C
//   3) x-lines:  grad = (Sd_x A, S_x B, S_x C) at the Gauss points, h = G_q grad (G_q the merged
//      metric), A <- Sd_x^T h_1, B <- S_x^T h_2, C <- S_x^T h_3, all in registers; the lattice
//      point that neighbouring cells of the batch share in x is summed here (in registers within
//      a pair, one shuffle between pairs), so from here on every point of the batch has one owner
//   4) y-lines:  A <- S_y^T A + Sd_y^T B,  C <- S_y^T C   (shared x-points: owner only)
//   5) z-lines:  out = S_z^T A + Sd_z^T C  into the output tile, one plain store per point, which
//      the TMA engine adds to dst (dst holds src on Dirichlet rows and 0 elsewhere beforehand).
// That is sixteen 1D contractions per line instead of twelve, in five phases instead of ten.
// Every thread owns the same line of two neighbouring cells (2c, 2c + 1) held as a float pair, so
// each contraction is a chain of packed FMAs and every shared-memory access moves 8 bytes; the
// cube paddings are those of the ten-phase kernel (same line access patterns).
//
// Input tile, output tile and (MS) the metric are single buffers: the next batch's rows are loaded
// once phase 1 has read the tile, the next batch's metric once phase 3 has read it, and the output
// tile is rewritten only after the TMA engine has read the previous batch's.  MS = 0 reads the
// metric at its point of use from L2 (the TMA engine prefetches each batch's metric into L2 one
// batch ahead); MS = 1 copies each batch's metric into shared memory with bulk copies (no L2
// prefetch).  Every mbarrier wait is bounded; on timeout the CTA sets the error word, drains its
// copies and returns.
#pragma once

#include "vmult_brick_tma2.cuh"

namespace mfx {

template <int N, int CB, int MS, int TB = 1, int MBF = 1, int PK = 0>
struct F5Shape {
  static constexpr int PP = CB / 2;
  static constexpr int LINES = PP * N * N;
  static constexpr int THREADS = (LINES + 31) / 32 * 32;
  static constexpr int CUBES = PP * BrickShape<N, CB, float>::CELL;  // float2 elements per cube
  static constexpr int METRIC = 6 * N * N * N * CB;                  // floats of one batch's metric
  // tile rows: 128-byte pitch for tensor copies, or packed at the box width (PK: untiled bulk copies)
  static constexpr int PITCH = PK ? TmaShape<N, CB>::BOX : TmaShape<N, CB>::PITCH;
  static constexpr int TILE = TmaShape<N, CB>::ROWS * PITCH;
  // TB input tiles and one output tile, MBF staged metric buffers (MS), three cubes, four mbarriers
  static constexpr size_t SMEM = (size_t)(TB + 1) * TILE * sizeof(float) +
                                 (MS ? (size_t)MBF * METRIC * sizeof(float) : 0) + 3 * (size_t)CUBES * sizeof(float2) +
                                 4 * sizeof(uint64_t);
  static_assert(32 % PP == 0, "the pairs of one line must share a warp (x-point shuffle)");
  static_assert((METRIC * sizeof(float)) % 16 == 0, "bulk copy size");
  static_assert((TILE * sizeof(float)) % 16 == 0 && (PITCH * sizeof(float)) % 16 == 0, "16-byte tile rows");
  static_assert(TB == 1 || TB == 2, "one or two input tiles");
  static_assert(MBF == 1 || MBF == 2, "one or two metric buffers");
};

// one bulk copy (no tensor map) global -> shared, completion on an mbarrier; both addresses 16-byte
// aligned, size a multiple of 16
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// dst[0 .. bytes / 4) += src[...] (untiled bulk reduce-add, bulk-group completion); both addresses
// 16-byte aligned, size a multiple of 16
__device__ __forceinline__ void bulk_reduce_add_f32(float* dst, const float* src, unsigned bytes) {
  asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f32 [%0], [%1], %2;\n" ::"l"(dst),
               "r"(smem_u32(src)), "r"(bytes)
               : "memory");
}

// L2 policy for data read once (the metric stream): evicted first, so that the vectors' lines stay
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
__device__ __forceinline__ void bulk_load_hint(void* dst, const void* src, unsigned bytes, uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ void prefetch_l2_bulk_hint(const void* p, unsigned bytes, uint64_t pol) {
  asm volatile("cp.async.bulk.prefetch.L2.global.L2::cache_hint [%0], %1, %2;\n" ::"l"(p), "r"(bytes), "l"(pol) : "memory");
}

// out = M1^T a + M2^T b
template <int N, int M1, int M2>
__device__ __forceinline__ void contract2_tt(const float2 (&a)[N], const float2 (&b)[N], float2 (&out)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const float m0 = (float)basis_entry<N, M1>(i);
    float2 s = __fmul2_rn(make_float2(m0, m0), a[0]);
#pragma unroll
    for (int j = 1; j < N; ++j) {
      const float mj = (float)basis_entry<N, M1>(j * N + i);
      s = __ffma2_rn(make_float2(mj, mj), a[j], s);
    }
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const float mj = (float)basis_entry<N, M2>(j * N + i);
      s = __ffma2_rn(make_float2(mj, mj), b[j], s);
    }
    out[i] = s;
  }
}

// row q of M times in
template <int N, int MAT>
__device__ __forceinline__ float2 row2(const float2 (&in)[N], int q) {
  const float m0 = (float)basis_entry<N, MAT>(q * N);
  float2 s = __fmul2_rn(make_float2(m0, m0), in[0]);
#pragma unroll
  for (int j = 1; j < N; ++j) {
    const float mj = (float)basis_entry<N, MAT>(q * N + j);
    s = __ffma2_rn(make_float2(mj, mj), in[j], s);
  }
  return s;
}

// acc[i] (+)= M[q][i] h  (column q of M^T)
template <int N, int MAT>
__device__ __forceinline__ void axpy_col2(float2 (&acc)[N], float2 h, int q, bool first) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const float m = (float)basis_entry<N, MAT>(q * N + i);
    acc[i] = first ? __fmul2_rn(make_float2(m, m), h) : __ffma2_rn(make_float2(m, m), h, acc[i]);
  }
}

// Even-odd form of the 1D contractions (used from N = 5 on, where it saves multiply-adds).  The 1D
// matrices are centro-symmetric (S: the nodal basis at Gauss points symmetric about 1/2) or
// centro-antisymmetric (Sd): M[N-1-i][N-1-j] = sg M[i][j] with sg = +1 / -1, and so are their
// transposes.  With e_j = v_j + v_{N-1-j}, d_j = v_j - v_{N-1-j} (j < N/2) and m = v_{N/2} (odd N):
//   out_i = E_i + O_i,  out_{N-1-i} = sg (E_i - O_i)   (i < N/2),
//   E_i = sum_j P_ij e_j + M_{i,N/2} m,  O_i = sum_j Q_ij d_j,  P_ij, Q_ij = (M_ij +- M_{i,N-1-j}) / 2,
// and the middle row of odd N is sum_j M_{N/2,j} e_j + M_{N/2,N/2} m (sg = +1) or sum_j M_{N/2,j} d_j
// (sg = -1).  T: apply the transpose.
template <int N>
constexpr bool kEvenOdd = N >= 5;

template <int N, int MAT, bool T>
__device__ __forceinline__ constexpr double eo_entry(int i, int j) {
  return T ? basis_entry<N, MAT>(j * N + i) : basis_entry<N, MAT>(i * N + j);
}

__device__ __forceinline__ float2 f2(double c) { return make_float2((float)c, (float)c); }

template <int N>
__device__ __forceinline__ void eo_split(const float2 (&v)[N], float2 (&e)[N / 2], float2 (&d)[N / 2]) {
#pragma unroll
  for (int j = 0; j < N / 2; ++j) {
    e[j] = __fadd2_rn(v[j], v[N - 1 - j]);
    d[j] = __ffma2_rn(make_float2(-1.0f, -1.0f), v[N - 1 - j], v[j]);
  }
}

// E_i (with the middle term) and O_i of row i < N/2
template <int N, int MAT, bool T>
__device__ __forceinline__ void eo_row(const float2 (&e)[N / 2], const float2 (&d)[N / 2], float2 m, int i, float2& E,
                                       float2& O) {
  constexpr int H = N / 2;
  E = __fmul2_rn(f2(0.5 * (eo_entry<N, MAT, T>(i, 0) + eo_entry<N, MAT, T>(i, N - 1))), e[0]);
  O = __fmul2_rn(f2(0.5 * (eo_entry<N, MAT, T>(i, 0) - eo_entry<N, MAT, T>(i, N - 1))), d[0]);
#pragma unroll
  for (int j = 1; j < H; ++j) {
    E = __ffma2_rn(f2(0.5 * (eo_entry<N, MAT, T>(i, j) + eo_entry<N, MAT, T>(i, N - 1 - j))), e[j], E);
    O = __ffma2_rn(f2(0.5 * (eo_entry<N, MAT, T>(i, j) - eo_entry<N, MAT, T>(i, N - 1 - j))), d[j], O);
  }
  if constexpr ((N & 1) != 0) E = __ffma2_rn(f2(eo_entry<N, MAT, T>(i, H)), m, E);
}

// the middle row of odd N
template <int N, int MAT, bool T>
__device__ __forceinline__ float2 eo_mid(const float2 (&e)[N / 2], const float2 (&d)[N / 2], float2 m) {
  constexpr int H = N / 2;
  if constexpr (MAT == MAT_S) {
    float2 s = __fmul2_rn(f2(eo_entry<N, MAT, T>(H, H)), m);
#pragma unroll
    for (int j = 0; j < H; ++j) s = __ffma2_rn(f2(eo_entry<N, MAT, T>(H, j)), e[j], s);
    return s;
  } else {
    float2 s = __fmul2_rn(f2(eo_entry<N, MAT, T>(H, 0)), d[0]);
#pragma unroll
    for (int j = 1; j < H; ++j) s = __ffma2_rn(f2(eo_entry<N, MAT, T>(H, j)), d[j], s);
    return s;
  }
}

// out = M v (T: M^T v) from a split input
template <int N, int MAT, bool T>
__device__ __forceinline__ void eo_apply(const float2 (&e)[N / 2], const float2 (&d)[N / 2], float2 m,
                                         float2 (&out)[N]) {
#pragma unroll
  for (int i = 0; i < N / 2; ++i) {
    float2 E, O;
    eo_row<N, MAT, T>(e, d, m, i, E, O);
    out[i] = __fadd2_rn(E, O);
    if constexpr (MAT == MAT_S)
      out[N - 1 - i] = __ffma2_rn(make_float2(-1.0f, -1.0f), O, E);  // E - O
    else
      out[N - 1 - i] = __ffma2_rn(make_float2(-1.0f, -1.0f), E, O);  // -(E - O)
  }
  if constexpr ((N & 1) != 0) out[N / 2] = eo_mid<N, MAT, T>(e, d, m);
}

// out = S^T a + Sd^T b (T) or S a + Sd b from split inputs: with X = E_S(a) + O_Sd(b) and
// Y = O_S(a) + E_Sd(b), out_i = X + Y and out_{N-1-i} = X - Y
template <int N, bool T>
__device__ __forceinline__ void eo_apply_s_sd(const float2 (&ea)[N / 2], const float2 (&da)[N / 2], float2 ma,
                                              const float2 (&eb)[N / 2], const float2 (&db)[N / 2], float2 mb,
                                              float2 (&out)[N]) {
#pragma unroll
  for (int i = 0; i < N / 2; ++i) {
    float2 Ea, Oa, Eb, Ob;
    eo_row<N, MAT_S, T>(ea, da, ma, i, Ea, Oa);
    eo_row<N, MAT_SD, T>(eb, db, mb, i, Eb, Ob);
    const float2 X = __fadd2_rn(Ea, Ob), Y = __fadd2_rn(Oa, Eb);
    out[i] = __fadd2_rn(X, Y);
    out[N - 1 - i] = __ffma2_rn(make_float2(-1.0f, -1.0f), Y, X);
  }
  if constexpr ((N & 1) != 0)
    out[N / 2] = __fadd2_rn(eo_mid<N, MAT_S, T>(ea, da, ma), eo_mid<N, MAT_SD, T>(eb, db, mb));
}

// The contractions of the phases, in even-odd form from N = 5 on
template <int N>
__device__ __forceinline__ void c2_s_sd(const float2 (&v)[N], float2 (&os)[N], float2 (&od)[N]) {  // S v, Sd v
  if constexpr (kEvenOdd<N>) {
    float2 e[N / 2], d[N / 2];
    eo_split<N>(v, e, d);
    eo_apply<N, MAT_S, false>(e, d, v[N / 2], os);
    eo_apply<N, MAT_SD, false>(e, d, v[N / 2], od);
  } else {
    contract2<N, MAT_S>(v, os);
    contract2<N, MAT_SD>(v, od);
  }
}
template <int N, int MAT, bool T>
__device__ __forceinline__ void c2_one(const float2 (&v)[N], float2 (&o)[N]) {  // M v or M^T v
  if constexpr (kEvenOdd<N>) {
    float2 e[N / 2], d[N / 2];
    eo_split<N>(v, e, d);
    eo_apply<N, MAT, T>(e, d, v[N / 2], o);
  } else if constexpr (T) {
    contract2_t<N, MAT>(v, o);
  } else {
    contract2<N, MAT>(v, o);
  }
}
template <int N>
__device__ __forceinline__ void c2_tt(const float2 (&a)[N], const float2 (&b)[N], float2 (&o)[N]) {  // S^T a + Sd^T b
  if constexpr (kEvenOdd<N>) {
    float2 ea[N / 2], da[N / 2], eb[N / 2], db[N / 2];
    eo_split<N>(a, ea, da);
    eo_split<N>(b, eb, db);
    eo_apply_s_sd<N, true>(ea, da, a[N / 2], eb, db, b[N / 2], o);
  } else {
    contract2_tt<N, MAT_S, MAT_SD>(a, b, o);
  }
}

// MS: metric staged in shared memory (1) or read from L2 (0); MB: CTAs per SM the registers are sized for;
// TB: input tiles (2: the next batch's rows are requested when a batch starts, 1: once phase 1 has read
// the tile); MBF: staged metric buffers (2: the next batch's metric is requested when a batch starts);
// EF: the metric stream carries the L2 evict-first policy
template <int N, int CB, int MS, int MB, int TB, int MBF, int EF, int PK = 0, bool BOXM = false>
__global__ void __launch_bounds__(F5Shape<N, CB, MS, TB, MBF, PK>::THREADS, MB)
    brick_vmult_f5_kernel(const __grid_constant__ TmaArgs<N> a) {
  static_assert(!BOXM || MS == 0, "box cells read the metric from global memory");
  using Sh = BrickShape<N, CB, float>;  // cube paddings of CB cells = paddings of CB / 2 float pairs
  using Tm = TmaShape<N, CB>;
  using Fs = F5Shape<N, CB, MS, TB, MBF, PK>;
  constexpr int PP = Fs::PP;
  constexpr int K = Sh::K, NP = Sh::NP, P2 = Sh::P2, CELL = Sh::CELL, N3 = N * N * N;
  constexpr int PITCH = Fs::PITCH, ROWS = Tm::ROWS, BOX = Tm::BOX;
  constexpr unsigned MBYTES = Fs::METRIC * 4u;
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* T0 = reinterpret_cast<float*>(smem_raw);  // input tile(s)
  float* O = T0 + TB * Fs::TILE;                    // output tile
  float* M0 = O + Fs::TILE;                         // MS: staged metric buffer(s), [6][N^3][CB] each
  float2* A = reinterpret_cast<float2*>(M0 + (MS ? MBF * Fs::METRIC : 0));
  float2* B = A + Fs::CUBES;
  float2* C = B + Fs::CUBES;
  // [0], [1]: input tiles, [2], [3]: metric buffers
  uint64_t* bars = reinterpret_cast<uint64_t*>(C + Fs::CUBES);

  const int t = threadIdx.x;
  const int c = t % PP;  // pair: cells 2c and 2c + 1 of the batch
  const int r = t / PP;
  const int f = r % N, s = r / N;
  const bool line_ok = t < Fs::LINES;
  const int xa2 = Sh::XSWAP ? s : f, xa3 = Sh::XSWAP ? f : s;
  const int xbase = c * CELL + xa3 * P2 + xa2 * NP;
  const int ybase = c * CELL + s * P2 + f;
  const int zbase = c * CELL + s * NP + f;
  const int zx = 2 * c * K + f;  // tile point of this thread's z-line in the first cell of the pair; + K for the second
  const int lane = t & 31;
  const bool tma_warp = (t >> 5) == Fs::THREADS / 32 - 1;  // the last warp (idle lanes) issues the copies
  // this thread's x-line of quadrature points in the metric of a batch (float2 units: cells 2c, 2c + 1)
  const int gq = (xa2 * N + xa3 * N * N) * PP + c;
  const uint64_t pol = (EF && tma_warp) ? policy_evict_first() : 0ull;

  if (t == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) mbar_init(&bars[i], 1);
    fence_mbar_init();
  }
  __syncthreads();

  auto issue_rows = [&](const BatchPos& pb, int buf) {
    const BatchInfo bi = batch_info_at<CB, K>(a, pb);
    fence_proxy_async();
    float* T = T0 + buf * Fs::TILE;
    if constexpr (PK) {
      // untiled bulk copies of the rows, clipped at the end of src: the whole 16-byte words inside src
      // by the copy engine, the last 0..3 points by plain loads, the rest of the box zero
      unsigned bytes = 0;
      for (int row = lane; row < ROWS; row += 32) {
        const int a2 = row % N, a3 = row / N;
        const int64_t g0 = (int64_t)((bi.gbase + a.Mx * (a2 + a.My * a3)) & ~3);
        const int len = (int)(a.n - g0 < BOX ? a.n - g0 : BOX);
        bytes += (unsigned)(len & ~3) * 4u;
      }
      bytes = __reduce_add_sync(0xffffffffu, bytes);
      if (lane == 0) mbar_arrive_expect_tx(&bars[buf], bytes);
      __syncwarp();
      for (int row = lane; row < ROWS; row += 32) {
        const int a2 = row % N, a3 = row / N;
        const int64_t g0 = (int64_t)((bi.gbase + a.Mx * (a2 + a.My * a3)) & ~3);
        const int len = (int)(a.n - g0 < BOX ? a.n - g0 : BOX);
        const int whole = len & ~3;
        float* dst = T + row * PITCH;
        if (whole > 0) bulk_load(dst, a.src + g0, (unsigned)whole * 4u, &bars[buf]);
        for (int x = whole; x < BOX; ++x) dst[x] = x < len ? a.src[g0 + x] : 0.0f;
      }
    } else {
      if (lane == 0) mbar_arrive_expect_tx(&bars[buf], ROWS * BOX * 4);
      __syncwarp();
      for (int row = lane; row < ROWS; row += 32) {
        const int a2 = row % N, a3 = row / N;
        tma_load_1d(T + row * PITCH, &a.tsrc, (bi.gbase + a.Mx * (a2 + a.My * a3)) & ~3, &bars[buf]);
      }
    }
  };
  // MS: the batch's metric in four bulk copies (lanes 0..3)
  auto issue_metric = [&](int bn, int buf) {
    constexpr unsigned CH = (MBYTES / 4 + 15u) & ~15u;
    if (lane == 0) mbar_arrive_expect_tx(&bars[2 + buf], MBYTES);
    __syncwarp();
    const unsigned off = lane * CH;
    if (lane < 4 && off < MBYTES) {
      char* d = reinterpret_cast<char*>(M0 + buf * Fs::METRIC) + off;
      const char* g = reinterpret_cast<const char*>(a.metric + (int64_t)bn * Fs::METRIC) + off;
      const unsigned n = off + CH <= MBYTES ? CH : MBYTES - off;
      if (EF)
        bulk_load_hint(d, g, n, &bars[2 + buf], pol);
      else
        bulk_load(d, g, n, &bars[2 + buf]);
    }
  };

  int it = 0;
  bool failed = false;
  // copies in flight that no wait has seen yet (bit i: mbarrier i), and the parity of the phase they
  // complete (bit i)
  unsigned pend = 0u, par = 0u;
  auto mark = [&](int i, bool on, unsigned parity) {
    pend = on ? (pend | (1u << i)) : (pend & ~(1u << i));
    par = (par & ~(1u << i)) | (parity << i);
  };
  BatchPos pos = batch_pos(a, blockIdx.x);
  if ((int)blockIdx.x < a.n_batches) {
    if (tma_warp) {
      issue_rows(pos, 0);
      if (MS) issue_metric(blockIdx.x, 0);
    }
    mark(0, true, 0u);
    mark(2, MS != 0, 0u);
  }

  for (int b = blockIdx.x; b < a.n_batches; b += gridDim.x, ++it) {
    const BatchInfo bi = batch_info_at<CB, K>(a, pos);
    const int m = bi.m;
    const bool act = line_ok && 2 * c < m;       // first cell of the pair valid
    const bool act1 = line_ok && 2 * c + 1 < m;  // second cell valid
    // pairs that hold the batch's last cell also own its last lattice point in x (a1 = K)
    const bool own_k = 2 * c == m - 1 || 2 * c + 1 == m - 1;
    const bool act45 = act && (f < K || own_k);
    const bool has_next = b + (int)gridDim.x < a.n_batches;
    const int zrow0 = bi.gbase + a.Mx * s;
    const bool ebnd = (s == 0 && (bi.eflags & 1)) || (s == K && (bi.eflags & 2));
    const bool lbnd0 = ebnd || (zx == 0 && bi.xlo) || (zx == bi.Wm - 1 && bi.xhi);
    const bool lbnd1 = ebnd || (zx + K == 0 && bi.xlo) || (zx + K == bi.Wm - 1 && bi.xhi);
    const bool zlo = (bi.eflags & 4) != 0, zhi = (bi.eflags & 8) != 0;

    const int rbuf = TB == 2 ? (it & 1) : 0;
    const unsigned rpar = TB == 2 ? ((it >> 1) & 1) : (it & 1);
    const int mbuf = MBF == 2 ? (it & 1) : 0;
    const unsigned mpar = MBF == 2 ? ((it >> 1) & 1) : (it & 1);
    float* T = T0 + rbuf * Fs::TILE;
    const float* Msm = M0 + mbuf * Fs::METRIC;
    // metric read from L2 (MS = 0): the TMA engine brings the next batch's metric into L2 (nothing waits
    // for it); with the staged metric the bulk copy alone measured faster (Q4 0.2585 -> 0.2503 ms, Q2
    // 0.3406 -> 0.3261 ms against an L2 prefetch two batches ahead)
    if (!MS && !BOXM && tma_warp && lane >= 4 && lane < 7) {
      const int bn = b + (int)gridDim.x;
      if (bn < a.n_batches) {
        constexpr unsigned CHUNK = (MBYTES / 3 + 15u) & ~15u;
        const unsigned off = (lane - 4) * CHUNK;
        if (off < MBYTES) {
          const char* g = reinterpret_cast<const char*>(a.metric + (int64_t)bn * Fs::METRIC) + off;
          const unsigned n = off + CHUNK <= MBYTES ? CHUNK : MBYTES - off;
          if (EF)
            prefetch_l2_bulk_hint(g, n, pol);
          else
            prefetch_l2_bulk(g, n);
        }
      }
    }
    // double buffers: the next batch's rows and metric go into the buffers the previous batch read
    // (phases 1 and 3 of the previous batch ended with barriers)
    if (TB == 2 && has_next) {
      if (tma_warp) {
        BatchPos next = pos;
        batch_advance(next, a);
        issue_rows(next, rbuf ^ 1);
      }
      mark(rbuf ^ 1, true, ((it + 1) >> 1) & 1);
    }
    if (MS && MBF == 2 && has_next) {
      if (tma_warp) issue_metric(b + (int)gridDim.x, mbuf ^ 1);
      mark(2 + (mbuf ^ 1), true, ((it + 1) >> 1) & 1);
    }
    {
      const bool ok = mbar_wait(&bars[rbuf], rpar);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      mark(rbuf, false, 0u);
    }
    // 1) z-lines of the input tile (Dirichlet points read as 0): A = S_z u, C = Sd_z u
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
      float2 od[N];
      c2_s_sd<N>(v, o, od);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        A[zbase + j * P2] = o[j];
        C[zbase + j * P2] = od[j];
      }
    }
    __syncthreads();
    // one input tile: it is free now, the next batch's rows
    if (TB == 1 && has_next) {
      if (tma_warp) {
        BatchPos next = pos;
        batch_advance(next, a);
        issue_rows(next, 0);
      }
      mark(0, true, (it + 1) & 1);
    }
    // 2) y-lines: A <- S_y A, B = Sd_y A, C <- S_y C
    if (act) {
      float2 v[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = A[ybase + j * NP];
      float2 od[N];
      c2_s_sd<N>(v, o, od);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        A[ybase + j * NP] = o[j];
        B[ybase + j * NP] = od[j];
      }
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = C[ybase + j * NP];
      c2_one<N, MAT_S, false>(v, o);
#pragma unroll
      for (int j = 0; j < N; ++j) C[ybase + j * NP] = o[j];
    }
    if (MS) {
      const bool ok = mbar_wait(&bars[2 + mbuf], mpar);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      mark(2 + mbuf, false, 0u);
    } else {
      __syncthreads();
    }
    // 3) x-lines: gradient at the Gauss points, metric, transposed x-contractions, in registers
    float2 ra[N], rb[N], rc[N];
#pragma unroll
    for (int i = 0; i < N; ++i) ra[i] = rb[i] = rc[i] = make_float2(0.0f, 0.0f);
    if (act) {
      float2 va[N], vb[N], vc[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        va[j] = A[xbase + j];
        vb[j] = B[xbase + j];
        vc[j] = C[xbase + j];
      }
      const float2* Gm = MS ? reinterpret_cast<const float2*>(Msm) + gq
                            : reinterpret_cast<const float2*>(a.metric + (int64_t)b * Fs::METRIC) + gq;
      // the merged metric at Gauss point q of this x-line: h = G grad
      // box cells: the metric on the line is w_q / w_0 times its first point's diagonal
      float2 D0 = make_float2(0.f, 0.f), D1 = D0, D2 = D0;
      if constexpr (BOXM) {
        D0 = __ldg(Gm);
        D1 = __ldg(Gm + 3 * N3 * PP);
        D2 = __ldg(Gm + 5 * N3 * PP);
      }
      auto qpoint = [&](int q, float2 u1, float2 u2, float2 u3, float2& h1, float2& h2, float2& h3) {
        if constexpr (BOXM) {
          const float2 rq = make_float2(a.wr[q], a.wr[q]);
          h1 = __fmul2_rn(__fmul2_rn(rq, D0), u1);
          h2 = __fmul2_rn(__fmul2_rn(rq, D1), u2);
          h3 = __fmul2_rn(__fmul2_rn(rq, D2), u3);
          return;
        }
        float2 G00, G01, G02, G11, G12, G22;
        if constexpr (MS != 0) {
          G00 = Gm[(0 * N3 + q) * PP]; G01 = Gm[(1 * N3 + q) * PP]; G02 = Gm[(2 * N3 + q) * PP];
          G11 = Gm[(3 * N3 + q) * PP]; G12 = Gm[(4 * N3 + q) * PP]; G22 = Gm[(5 * N3 + q) * PP];
        } else {
          G00 = __ldg(Gm + (0 * N3 + q) * PP); G01 = __ldg(Gm + (1 * N3 + q) * PP);
          G02 = __ldg(Gm + (2 * N3 + q) * PP); G11 = __ldg(Gm + (3 * N3 + q) * PP);
          G12 = __ldg(Gm + (4 * N3 + q) * PP); G22 = __ldg(Gm + (5 * N3 + q) * PP);
        }
        h1 = __ffma2_rn(G02, u3, __ffma2_rn(G01, u2, __fmul2_rn(G00, u1)));
        h2 = __ffma2_rn(G12, u3, __ffma2_rn(G11, u2, __fmul2_rn(G01, u1)));
        h3 = __ffma2_rn(G22, u3, __ffma2_rn(G12, u2, __fmul2_rn(G02, u1)));
      };
      if constexpr (kEvenOdd<N>) {
        // gradient at all Gauss points of the line, h in place, then the transposed contractions
        float2 u1[N], u2[N], u3[N];
        c2_one<N, MAT_SD, false>(va, u1);
        c2_one<N, MAT_S, false>(vb, u2);
        c2_one<N, MAT_S, false>(vc, u3);
#pragma unroll
        for (int q = 0; q < N; ++q) {
          float2 h1, h2, h3;
          qpoint(q, u1[q], u2[q], u3[q], h1, h2, h3);
          u1[q] = h1;
          u2[q] = h2;
          u3[q] = h3;
        }
        c2_one<N, MAT_SD, true>(u1, ra);
        c2_one<N, MAT_S, true>(u2, rb);
        c2_one<N, MAT_S, true>(u3, rc);
      } else {
#pragma unroll
        for (int q = 0; q < N; ++q) {
          float2 h1, h2, h3;
          qpoint(q, row2<N, MAT_SD>(va, q), row2<N, MAT_S>(vb, q), row2<N, MAT_S>(vc, q), h1, h2, h3);
          axpy_col2<N, MAT_SD>(ra, h1, q, q == 0);
          axpy_col2<N, MAT_S>(rb, h2, q, q == 0);
          axpy_col2<N, MAT_S>(rc, h3, q, q == 0);
        }
      }
    }
    // the x-point shared by cells 2c - 1 and 2c (pair c - 1's second cell, lane - 1) and the one
    // shared by cells 2c and 2c + 1 (this pair): summed into the higher cell's a1 = 0 node
    {
      const float ua = __shfl_up_sync(0xffffffffu, ra[K].y, 1);
      const float ub = __shfl_up_sync(0xffffffffu, rb[K].y, 1);
      const float uc = __shfl_up_sync(0xffffffffu, rc[K].y, 1);
      if (c > 0) {
        ra[0].x += ua;
        rb[0].x += ub;
        rc[0].x += uc;
      }
      if (act1) {
        ra[0].y += ra[K].x;
        rb[0].y += rb[K].x;
        rc[0].y += rc[K].x;
      }
    }
    if (act) {
#pragma unroll
      for (int j = 0; j < N; ++j) {
        A[xbase + j] = ra[j];
        B[xbase + j] = rb[j];
        C[xbase + j] = rc[j];
      }
    }
    __syncthreads();
    // one metric buffer: it is free now, the next batch's metric
    if (MS && MBF == 1 && has_next) {
      if (tma_warp) issue_metric(b + (int)gridDim.x, 0);
      mark(2, true, (it + 1) & 1);
    }
    // 4) y-lines: A <- S_y^T A + Sd_y^T B, C <- S_y^T C
    if (act45) {
      float2 va[N], vb[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        va[j] = A[ybase + j * NP];
        vb[j] = B[ybase + j * NP];
      }
      c2_tt<N>(va, vb, o);
#pragma unroll
      for (int j = 0; j < N; ++j) A[ybase + j * NP] = o[j];
#pragma unroll
      for (int j = 0; j < N; ++j) va[j] = C[ybase + j * NP];
      c2_one<N, MAT_S, true>(va, o);
#pragma unroll
      for (int j = 0; j < N; ++j) C[ybase + j * NP] = o[j];
    }
    // the output tile was last read by the previous batch's reduce-adds
    if (tma_warp) bulk_wait_read<0>();
    __syncthreads();
    // 5) z-lines: out = S_z^T A + Sd_z^T C into the output tile (Dirichlet points 0); the TMA warp
    //    clears the points of each tile row outside the batch
    if (act45) {
      float2 va[N], vc[N], o[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        va[j] = A[zbase + j * P2];
        vc[j] = C[zbase + j * P2];
      }
      c2_tt<N>(va, vc, o);
      const bool w0 = f < K || 2 * c == m - 1;
      const bool w1 = act1 && (f < K || 2 * c + 1 == m - 1);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        if (lbnd0) o[j].x = 0.0f;
        if (lbnd1) o[j].y = 0.0f;
      }
      if (zlo) o[0] = make_float2(0.0f, 0.0f);
      if (zhi) o[K] = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const int g = zrow0 + a.Mx * a.My * j;
        float* row = O + (j * N + s) * PITCH + (g & 3) + zx;
        if (w0) row[0] = o[j].x;
        if (w1) row[K] = o[j].y;
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
    fence_proxy_async();
    __syncthreads();
    // reduce-add the output rows into dst (one bulk group per lane and batch)
    if (tma_warp) {
      for (int row = lane; row < ROWS; row += 32) {
        const int a2 = row % N, a3 = row / N;
        const int g0 = (bi.gbase + a.Mx * (a2 + a.My * a3)) & ~3;
        if constexpr (PK) {
          // the whole 16-byte words inside dst by the copy engine, the last 0..3 points by atomics
          const int len = (int)(a.n - g0 < BOX ? a.n - g0 : BOX);
          const int whole = len & ~3;
          if (whole > 0) bulk_reduce_add_f32(a.dst + g0, O + row * PITCH, (unsigned)whole * 4u);
          for (int x = whole; x < len; ++x) atomicAdd(a.dst + g0 + x, O[row * PITCH + x]);
        } else {
          tma_reduce_add_1d(&a.tdst, g0, O + row * PITCH);
        }
      }
      bulk_commit();
    }
    batch_advance(pos, a);
  }
  if (tma_warp) bulk_wait_all();
  if (failed && tma_warp && lane == 0) {
    atomicExch(a.err, 1);
    // drain the copies that may still be in flight before the CTA ends (bounded waits)
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (pend >> i & 1u) mbar_wait(&bars[i], par >> i & 1u);
  }
}

}  // namespace mfx
