// Host launcher of the vmult kernels for one degree (included by vmult_k*.cu): picks the kernel for the
// mesh type, precision and degree (structured row batches, per-cell index tables, tensor-product
// hanging constraints) for the cell loop of the matrix-free operator (Sec. 3.6).
#pragma once

#include <algorithm>
#include <string>
#include <type_traits>

#include "mfx_internal.h"
#include "vmult.cuh"
#include "vmult_brick.cuh"
#include "vmult_brick_tma.cuh"
#include "vmult_brick_df.cuh"
#include "vmult_brick_tma2.cuh"
#include "vmult_brick_f5.cuh"
#include "vmult_cell5.cuh"
#include "vmult_octree2.cuh"

namespace mfx {

int device_sm_count();

// The kernels use the build-time tables; check that they match the operator's tables
// (computed at run time by the same routines) bit for bit.
template <int N>
mfx_status prepare_vmult_n(const mfx_op* op) {
  for (int i = 0; i < N * N; ++i)
    if (BasisConst<N>::S(i) != op->basis.S[i] || BasisConst<N>::D(i) != op->basis.D[i] ||
        BasisConst<N>::Sd(i) != op->basis.Sd[i])
      return set_error(MFX_EUNSUPPORTED, "build-time basis tables differ from the run-time ones");
  return MFX_OK;
}

template <int N, typename Real>
static void fill_vmult_args(const mfx_op* op, VmultArgs<N, Real>* a) {
  a->metric = std::is_same<Real, double>::value ? (const Real*)op->d_metric64 : (const Real*)op->d_metric32;
  a->n_cells = op->n_cells;
  a->cell_list = nullptr;
  a->n_list = 0;
  a->cell_dofs = op->d_cell_dofs;
  a->cptr = op->d_cptr;
  a->cmaster = op->d_cmaster;
  a->cweight = std::is_same<Real, double>::value ? (const Real*)op->d_cweight64 : (const Real*)op->d_cweight32;
  a->cmask = op->d_cmask;
  a->n_dofs = op->n_dofs;
  a->hface = op->d_hface;
  a->hedge = op->d_hedge;
  a->hoff = op->d_hoff;
  a->hdofs = op->d_hdofs;
  a->box = op->d_box32;
  for (int q = 0; q < N; ++q) a->wq[q] = (Real)op->basis.wq[q];
  for (int c = 0; c < 2; ++c)
    for (int b = 0; b < N; ++b)
      for (int m = 0; m < N; ++m)
        a->P[c * N * N + b * N + m] = (Real)lagrange_value(N, op->basis.gll, m, 0.5 * (c + op->basis.gll[b]));
}

// One launch of the per-cell kernel over all cells, or over a cell list (prologue: dst = src on the
// constrained rows and 0 elsewhere, before the first launch of a vmult).
template <int N, typename Real, bool HANG, bool BOX = false>
static mfx_status run_vmult_h(const mfx_op* op, const Real* src, Real* dst, cudaStream_t s, const int32_t* skip,
                              const int32_t* list, int64_t n_list, bool prologue) {
  using Sh = VmultShape<N>;
  static int blocks_per_sm = -1;
  // three cubes per cell, the coarse values of hanging faces and edges, and (five-phase kernel, small n)
  // the interpolation scratch
  const size_t hb = HANG ? (size_t)Sh::CB * (6 * N * N + 12 * N) : 0;
  const size_t smem = (3 * (size_t)Sh::CB * Sh::CELL + hb + (Cell5Scratch<N>::OWN ? hb : 0)) * sizeof(Real);
  // FP32: the five-phase kernel except at k = 7 (measured on octrees refined twice, ms, ten / five phases:
  // k = 1 0.0209 / 0.0204, k = 2 0.0276 / 0.0276, k = 4 0.0890 / 0.0859, k = 5 0.1353 / 0.1289, k = 6
  // 0.2177 / 0.2128, k = 7 0.1666 / 0.1705, k = 8 0.2570 / 0.2307); FP64: the ten-phase kernel (the
  // five-phase one spills at the 80-register bound of the hanging variant: k = 4 0.750 / 0.914)
  constexpr bool five = sizeof(Real) == 4 && N != 8;
  static_assert(!BOX || five, "the box-cell metric is read by the FP32 five-phase kernel only");
  auto kern = five ? vmult5_kernel<N, Real, HANG, BOX> : vmult_kernel<N, Real, HANG>;
  if (blocks_per_sm < 0) {
    MFX_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int b = 0;
    MFX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, Sh::THREADS, smem));
    blocks_per_sm = b > 0 ? b : 1;
  }
  VmultArgs<N, Real> a;
  fill_vmult_args<N, Real>(op, &a);
  a.skip = skip;
  a.cell_list = list;
  a.n_list = n_list;
  const int sms = device_sm_count();
  if (prologue) {
    int pb = (int)std::min<int64_t>((op->n_dofs + 255) / 256, (int64_t)sms * 8);
    if (pb < 1) pb = 1;
    vmult_prologue<N, Real><<<pb, 256, 0, s>>>(a, src, dst);
  }
  const int64_t nbatch = ((list ? n_list : op->n_cells) + Sh::CB - 1) / Sh::CB;
  if (nbatch > 0) {
    const int grid = (int)std::min<int64_t>(nbatch, (int64_t)sms * blocks_per_sm);
    kern<<<grid, Sh::THREADS, smem, s>>>(a, src, dst);
  }
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

// Hanging constraints in tensor-product form where they pay (k >= kTensorHangMinDegree), per-node master
// expansion otherwise.
template <int N, typename Real>
static mfx_status run_vmult(const mfx_op* op, const Real* src, Real* dst, cudaStream_t s, const int32_t* skip) {
  if constexpr (sizeof(Real) == 4 && N != 8) {
    if (op->box32) {
      if (N - 1 >= kTensorHangMinDegree && op->n_hanging > 0 && op->d_cells_hang) {
        mfx_status st =
            run_vmult_h<N, Real, false, true>(op, src, dst, s, skip, op->d_cells_plain, op->n_cells_plain, true);
        if (st != MFX_OK) return st;
        return run_vmult_h<N, Real, true, true>(op, src, dst, s, skip, op->d_cells_hang, op->n_cells_hang, false);
      }
      return run_vmult_h<N, Real, false, true>(op, src, dst, s, skip, nullptr, 0, true);
    }
  }
  if (N - 1 >= kTensorHangMinDegree && op->n_hanging > 0 && op->d_cells_hang) {
    // cells without hanging faces or edges in the plain kernel, the rest in the tensor-product one, one
    // launch after the other (side by side on two streams with grids split by work share measured slower:
    // 0.089 -> 0.111 ms on 16^3 coarse cells refined twice, Q4)
    mfx_status st = run_vmult_h<N, Real, false>(op, src, dst, s, skip, op->d_cells_plain, op->n_cells_plain, true);
    if (st != MFX_OK) return st;
    return run_vmult_h<N, Real, true>(op, src, dst, s, skip, op->d_cells_hang, op->n_cells_hang, false);
  }
  return run_vmult_h<N, Real, false>(op, src, dst, s, skip, nullptr, 0, true);
}

template <int N, typename Real, int CB>
static mfx_status run_brick(const mfx_op* op, const Real* src, Real* dst, cudaStream_t s, const int32_t* skip) {
  using Sh = BrickShape<N, CB, Real>;
  static int blocks_per_sm = -1;
  const size_t smem = Sh::SMEM;
  // FP64 in double-float arithmetic (same shared memory: a float pair per value)
  static_assert(std::is_same<Real, double>::value, "the FP32 structured path is run_brick_tma2");
  auto kern = brick_vmult_df_kernel<N, CB>;
  if (blocks_per_sm < 0) {
    MFX_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int b = 0;
    MFX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, Sh::THREADS, smem));
    blocks_per_sm = b > 0 ? b : 1;
  }
  if (op->metric_cb != CB) return set_error(MFX_EINVAL, "metric layout does not match the kernel");
  BrickArgs<N, Real> a;
  a.metric = std::is_same<Real, double>::value ? (const Real*)op->d_metric64 : (const Real*)op->d_metric32;
  a.nx = op->nx;
  a.ny = op->ny;
  a.nz = op->nz;
  a.nchunk = (op->nx + CB - 1) / CB;
  a.Mx = op->k * op->nx + 1;
  a.My = op->k * op->ny + 1;
  a.Mz = op->k * op->nz + 1;
  a.n_batches = (int64_t)a.nchunk * op->ny * op->nz;
  a.skip = skip;
  a.dmask = op->dirichlet;
  MFX_CUDA_TRY(cudaMemsetAsync(dst, 0, sizeof(Real) * op->n_dofs, s));
  const int grid = (int)std::min<int64_t>(a.n_batches, (int64_t)device_sm_count() * blocks_per_sm);
  kern<<<grid, Sh::THREADS, smem, s>>>(a, src, dst);
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

template <int N>
int brick_cells_per_batch() { return BrickCB<N>::value; }

template <int N>
int octree_pair_cells() { return OctreePairFor<N>::value ? BrickCB<N>::value : 0; }

// Batch sizes (cells per batch) compiled for degree N - 1, default first; the operator picks one
// by timing (autotuning) or takes the caller's choice.
template <int N>
int brick_cells_candidates(int* out) {
  out[0] = BrickCB<N>::value;
  if (BrickCB<N>::ALT > 0) {
    out[1] = BrickCB<N>::ALT;
    return 2;
  }
  return 1;
}

// Initial dst of the reduce-add kernels, in one pass: src on the Dirichlet DoFs (faces in dmask, the
// identity rows of the operator), 0 elsewhere.  One warp per lattice row (J, L).
template <typename Real>
__global__ void init_rows_kernel(int Mx, int My, int Mz, uint32_t dmask, const Real* __restrict__ src,
                                 Real* __restrict__ dst) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const int rows = My * Mz;
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < rows; row += warps) {
    const int J = row % My, L = row / My;
    const int64_t base = (int64_t)Mx * row;
    const bool whole = ((dmask & 4u) && J == 0) || ((dmask & 8u) && J == My - 1) || ((dmask & 16u) && L == 0) ||
                       ((dmask & 32u) && L == Mz - 1);
    for (int I = lane; I < Mx; I += 32) {
      const bool d = whole || ((dmask & 1u) && I == 0) || ((dmask & 2u) && I == Mx - 1);
      dst[base + I] = d ? src[base + I] : Real(0);
    }
  }
}

// The grid size as a step of batch positions (chunk, y, z) for batch_advance.
template <int N>
static void set_batch_steps(TmaArgs<N>* a, int grid) {
  const int row = grid / a->nchunk;
  a->step_chunk = grid - row * a->nchunk;
  a->step_y = row % a->ny;
  a->step_z = row / a->ny;
}

static int init_rows_grid(int rows) { return std::max(1, std::min((rows + 7) / 8, device_sm_count() * 16)); }

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static mfx_status encode_1d_map(CUtensorMap* map, const void* ptr, int64_t n, int box) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    MFX_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (!p || q != cudaDriverEntryPointSuccess) return set_error(MFX_ECUDA, "cuTensorMapEncodeTiled unavailable");
    fn = (EncodeTiledFn)p;
  }
  if (((uintptr_t)ptr & 15) != 0) return set_error(MFX_EINVAL, "vectors must be 16-byte aligned");
  const cuuint64_t dim[1] = {(cuuint64_t)n};
  // rank 1 has no strides, but the driver expects a valid array
  const cuuint64_t strides[1] = {(cuuint64_t)n * sizeof(float)};
  const cuuint32_t boxd[1] = {(cuuint32_t)box};
  const cuuint32_t estr[1] = {1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 1, const_cast<void*>(ptr), dim, strides, boxd, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(MFX_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return MFX_OK;
}

template <int N, int CB, bool BOXM = false>
static mfx_status run_brick_tma2(const mfx_op* op, const float* src, float* dst, cudaStream_t s, const int32_t* skip) {
  using Ps = PairShape<N, CB>;
  using Tm = TmaShape<N, CB>;
  static int blocks_per_sm = -1;
  const size_t smem = Ps::SMEM;
  auto kern = brick_vmult_tma2_kernel<N, CB, BOXM>;
  if (blocks_per_sm < 0) {
    MFX_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int b = 0;
    MFX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, Ps::THREADS, smem));
    blocks_per_sm = b > 0 ? b : 1;
  }
  if (op->metric_cb != CB) return set_error(MFX_EINVAL, "metric layout does not match the kernel");
  TmaArgs<N> a;
  mfx_status st = encode_1d_map(&a.tsrc, src, op->n_dofs, Tm::BOX);
  if (st != MFX_OK) return st;
  st = encode_1d_map(&a.tdst, dst, op->n_dofs, Tm::BOX);
  if (st != MFX_OK) return st;
  a.metric = op->d_metric32;
  a.nx = op->nx;
  a.ny = op->ny;
  a.nz = op->nz;
  a.nchunk = (op->nx + CB - 1) / CB;
  a.Mx = op->k * op->nx + 1;
  a.My = op->k * op->ny + 1;
  a.Mz = op->k * op->nz + 1;
  a.n_batches = a.nchunk * op->ny * op->nz;
  a.err = op->d_err;
  a.skip = skip;
  a.dmask = op->dirichlet;
  for (int q = 0; q < N; ++q) a.wr[q] = (float)(op->basis.wq[q] / op->basis.wq[0]);
  const int rows = a.My * a.Mz;
  init_rows_kernel<float><<<init_rows_grid(rows), 256, 0, s>>>(a.Mx, a.My, a.Mz, a.dmask, src, dst);
  const int grid = std::min(a.n_batches, device_sm_count() * blocks_per_sm);
  set_batch_steps(&a, grid);
  kern<<<grid, Ps::THREADS, smem, s>>>(a);
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

// The five-phase FP32 kernel (vmult_brick_f5.cuh) for degrees 1..4; MS: metric staged in shared
// memory (1) or read from L2 at its point of use (0).
template <int N>
struct F5For {
  static constexpr bool value = N >= 2 && N <= 5;
};

// Buffering of the five-phase kernel: one input tile and one staged metric buffer, no L2 policy.
// Measured on 64^3 Q4 / 86^3 Q3 / 128^3 Q2 against two input tiles, two metric buffers and the
// evict-first policy on the metric stream: the tiles and the policy within 2 % either way, the second
// metric buffer 26 % slower at Q2 (fewer CTAs per SM).
template <int N, int CB, int MS>
struct F5Config {
  static constexpr int TB = 1;
  static constexpr int MBF = 1;
  static constexpr int EF = 0;
  // tile rows packed at the box width and moved by untiled bulk copies (clipped at the vector end) where
  // the smaller tiles give one more CTA per SM: staged metric at Q4 with 8 cells per batch (five CTAs
  // instead of four: 64^3 0.2409 -> 0.2332 ms) and at Q3 with 16 (86^3 0.2912 -> 0.2831 ms); elsewhere
  // measured slower (Q4 16 cells 0.2563 -> 0.2735, Q3 8 cells 0.3179 -> 0.3322, Q2 32 cells 0.3261 ->
  // 0.3485 ms)
  static constexpr int PK = (MS && ((N == 5 && CB == 8) || (N == 4 && CB == 16))) ? 1 : 0;
};

template <int N, int CB, int MS, bool BOXM = false>
static mfx_status run_brick_f5(const mfx_op* op, const float* src, float* dst, cudaStream_t s, const int32_t* skip) {
  using Cf = F5Config<N, CB, MS>;
  constexpr int PK = Cf::PK;
  using Fs = F5Shape<N, CB, MS, Cf::TB, Cf::MBF, PK>;
  using Tm = TmaShape<N, CB>;
  // resident CTAs per SM the register budget is sized for: about 672 threads per SM, fewer when the
  // shared memory bounds them (228 KB per SM, 1 KB of it reserved per CTA)
  constexpr int MB0 = 672 / Fs::THREADS > 0 ? 672 / Fs::THREADS : 1;
  constexpr int MBS = (int)((228u * 1024u) / (Fs::SMEM + 1024u)) > 0 ? (int)((228u * 1024u) / (Fs::SMEM + 1024u)) : 1;
  constexpr int MB = MB0 < MBS ? MB0 : MBS;
  static int blocks_per_sm = -1;
  const size_t smem = Fs::SMEM;
  auto kern = brick_vmult_f5_kernel<N, CB, MS, MB, Cf::TB, Cf::MBF, Cf::EF, PK, BOXM>;
  if (blocks_per_sm < 0) {
    MFX_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int b = 0;
    MFX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, Fs::THREADS, smem));
    blocks_per_sm = b > 0 ? b : 1;
  }
  if (op->metric_cb != CB) return set_error(MFX_EINVAL, "metric layout does not match the kernel");
  TmaArgs<N> a;
  mfx_status st = encode_1d_map(&a.tsrc, src, op->n_dofs, Tm::BOX);
  if (st != MFX_OK) return st;
  st = encode_1d_map(&a.tdst, dst, op->n_dofs, Tm::BOX);
  if (st != MFX_OK) return st;
  a.metric = op->d_metric32;
  a.src = src;
  a.dst = dst;
  a.n = op->n_dofs;
  a.nx = op->nx;
  a.ny = op->ny;
  a.nz = op->nz;
  a.nchunk = (op->nx + CB - 1) / CB;
  a.Mx = op->k * op->nx + 1;
  a.My = op->k * op->ny + 1;
  a.Mz = op->k * op->nz + 1;
  a.n_batches = a.nchunk * op->ny * op->nz;
  a.err = op->d_err;
  a.skip = skip;
  a.dmask = op->dirichlet;
  for (int q = 0; q < N; ++q) a.wr[q] = (float)(op->basis.wq[q] / op->basis.wq[0]);
  const int rows = a.My * a.Mz;
  init_rows_kernel<float><<<init_rows_grid(rows), 256, 0, s>>>(a.Mx, a.My, a.Mz, a.dmask, src, dst);
  const int grid = std::min(a.n_batches, device_sm_count() * blocks_per_sm);
  set_batch_steps(&a, grid);
  kern<<<grid, Fs::THREADS, smem, s>>>(a);
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

template <int N, int CB>
static mfx_status run_brick_f32(const mfx_op* op, const float* src, float* dst, cudaStream_t s, const int32_t* skip) {
  // box cells: the chosen kernel's variant that reads three entries of each line's metric (the staged
  // five-phase kernel in its unstaged form: there is nothing left to stage)
  if (op->box32) {
    if constexpr (F5For<N>::value)
      if (op->f32_kernel == MFX_KERNEL_FIVE_PHASE || op->f32_kernel == MFX_KERNEL_FIVE_PHASE_STAGED)
        return run_brick_f5<N, CB, 0, true>(op, src, dst, s, skip);
    return run_brick_tma2<N, CB, true>(op, src, dst, s, skip);
  }
  if constexpr (F5For<N>::value) {
    if (op->f32_kernel == MFX_KERNEL_FIVE_PHASE) return run_brick_f5<N, CB, 0>(op, src, dst, s, skip);
    if (op->f32_kernel == MFX_KERNEL_FIVE_PHASE_STAGED) return run_brick_f5<N, CB, 1>(op, src, dst, s, skip);
  }
  return run_brick_tma2<N, CB>(op, src, dst, s, skip);
}

template <int N>
int brick_kernel_candidates(int* out) {
  int n = 0;
  out[n++] = MFX_KERNEL_TEN_PHASE;
  if (F5For<N>::value) {
    out[n++] = MFX_KERNEL_FIVE_PHASE;
    out[n++] = MFX_KERNEL_FIVE_PHASE_STAGED;
  }
  return n;
}

template <int N, int CB, bool BOX>
static mfx_status run_octree_pair(const mfx_op* op, const float* src, float* dst, cudaStream_t s,
                                  const int32_t* skip) {
  using Ps = PairShape<N, CB>;
  using Os = OctreePairShape<N, CB>;
  static int blocks_per_sm = -1;
  const size_t smem = Os::SMEM;
  auto kern = octree_vmult_pair_kernel<N, CB, BOX>;
  if (blocks_per_sm < 0) {
    MFX_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int b = 0;
    MFX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, Ps::THREADS, smem));
    blocks_per_sm = b > 0 ? b : 1;
  }
  if (op->metric_cb32 != CB) return set_error(MFX_EINVAL, "metric layout does not match the kernel");
  VmultArgs<N, float> pa;
  fill_vmult_args<N, float>(op, &pa);
  pa.skip = skip;
  const int sms = device_sm_count();
  int pb = (int)std::min<int64_t>((op->n_dofs + 255) / 256, (int64_t)sms * 8);
  if (pb < 1) pb = 1;
  vmult_prologue<N, float><<<pb, 256, 0, s>>>(pa, src, dst);
  OctreePairArgs<N> a;
  a.metric = op->d_metric32;
  a.cell_dofs = op->d_cell_dofs;
  a.cptr = op->d_cptr;
  a.cmaster = op->d_cmaster;
  a.cweight = op->d_cweight32;
  a.n_cells = op->n_cells;
  a.n_batches = (int)((op->n_cells + CB - 1) / CB);
  a.skip = skip;
  a.box = op->d_box32;
  for (int q = 0; q < N; ++q) a.wq[q] = (float)op->basis.wq[q];
  if (a.n_batches > 0) {
    const int grid = std::min(a.n_batches, sms * blocks_per_sm);
    kern<<<grid, Ps::THREADS, smem, s>>>(a, src, dst);
  }
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

template <int N>
mfx_status launch_vmult_n(const mfx_op* op, mfx_prec prec, const void* src, void* dst, cudaStream_t s,
                          const int32_t* skip) {
  constexpr int CB0 = BrickCB<N>::value;
  constexpr int CB1 = BrickCB<N>::ALT > 0 ? BrickCB<N>::ALT : CB0;
  if (prec == MFX_F64) {
    if (op->structured) {
      if (CB1 != CB0 && op->metric_cb == CB1) return run_brick<N, double, CB1>(op, (const double*)src, (double*)dst, s, skip);
      return run_brick<N, double, CB0>(op, (const double*)src, (double*)dst, s, skip);
    }
    return run_vmult<N, double>(op, (const double*)src, (double*)dst, s, skip);
  }
  if (op->structured && !op->percell32) {
    if (CB1 != CB0 && op->metric_cb == CB1) return run_brick_f32<N, CB1>(op, (const float*)src, (float*)dst, s, skip);
    return run_brick_f32<N, CB0>(op, (const float*)src, (float*)dst, s, skip);
  }
  // k = 1 box cells: one thread per cell, octant groups gathered and scattered once per node
  if constexpr (N == 2)
    if (op->box32 && op->q1_split) return launch_octree_q1_box(op, (const float*)src, (float*)dst, s, skip);
  // the paired octree kernel where the FP32 metric is laid out for it (k = 1; k = 8 without hanging nodes)
  if constexpr (OctreePairFor<N>::value)
    if (op->metric_cb32 > 0)
      return op->box32 ? run_octree_pair<N, CB0, true>(op, (const float*)src, (float*)dst, s, skip)
                       : run_octree_pair<N, CB0, false>(op, (const float*)src, (float*)dst, s, skip);
  return run_vmult<N, float>(op, (const float*)src, (float*)dst, s, skip);
}

}  // namespace mfx
