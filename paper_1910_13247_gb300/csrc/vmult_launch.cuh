// Host launcher of the vmult kernels for one degree (included by vmult_k*.cu).
#pragma once

#include <algorithm>
#include <type_traits>

#include "mfx_internal.h"
#include "vmult.cuh"
#include "vmult_brick.cuh"

namespace mfx {

int device_sm_count();

// Upload the 1D matrices of degree N - 1 into this translation unit's constant memory on the
// current device (once per device; the tables depend only on the degree).
template <int N>
mfx_status prepare_vmult_n(const mfx_op* op) {
  static bool done[64] = {false};
  int dev = 0;
  MFX_CUDA_TRY(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && done[dev]) return MFX_OK;
  float b32[2 * 81] = {0};
  double b64[2 * 81] = {0};
  for (int i = 0; i < N * N; ++i) {
    b64[i] = op->basis.S[i];
    b64[81 + i] = op->basis.D[i];
    b32[i] = (float)op->basis.S[i];
    b32[81 + i] = (float)op->basis.D[i];
  }
  MFX_CUDA_TRY(cudaMemcpyToSymbol(c_basis32, b32, sizeof(b32)));
  MFX_CUDA_TRY(cudaMemcpyToSymbol(c_basis64, b64, sizeof(b64)));
  if (dev >= 0 && dev < 64) done[dev] = true;
  return MFX_OK;
}

template <int N, typename Real>
static void fill_vmult_args(const mfx_op* op, VmultArgs<N, Real>* a) {
  a->metric = std::is_same<Real, double>::value ? (const Real*)op->d_metric64 : (const Real*)op->d_metric32;
  a->n_cells = op->n_cells;
  a->nx = op->nx;
  a->ny = op->ny;
  a->nz = op->nz;
  a->k = op->k;
  a->Mx = op->k * op->nx + 1;
  a->My = op->k * op->ny + 1;
  a->Mz = op->k * op->nz + 1;
  a->cell_dofs = op->d_cell_dofs;
  a->cptr = op->d_cptr;
  a->cmaster = op->d_cmaster;
  a->cweight = std::is_same<Real, double>::value ? (const Real*)op->d_cweight64 : (const Real*)op->d_cweight32;
  a->cmask = op->d_cmask;
  a->n_dofs = op->n_dofs;
}

template <int N, typename Real, bool STRUCT>
static mfx_status run_vmult(const mfx_op* op, const Real* src, Real* dst, cudaStream_t s, const int32_t* skip) {
  using Sh = VmultShape<N>;
  static int blocks_per_sm = -1;
  const size_t smem = 3 * (size_t)Sh::CB * Sh::CELL * sizeof(Real);
  auto kern = vmult_kernel<N, Real, STRUCT>;
  if (blocks_per_sm < 0) {
    MFX_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int b = 0;
    MFX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, Sh::THREADS, smem));
    blocks_per_sm = b > 0 ? b : 1;
  }
  VmultArgs<N, Real> a;
  fill_vmult_args<N, Real>(op, &a);
  a.skip = skip;
  const int sms = device_sm_count();
  int pb = (int)std::min<int64_t>((op->n_dofs + 255) / 256, (int64_t)sms * 8);
  if (pb < 1) pb = 1;
  vmult_prologue<N, Real, STRUCT><<<pb, 256, 0, s>>>(a, src, dst);
  const int64_t nbatch = (op->n_cells + Sh::CB - 1) / Sh::CB;
  if (nbatch > 0) {
    const int grid = (int)std::min<int64_t>(nbatch, (int64_t)sms * blocks_per_sm);
    kern<<<grid, Sh::THREADS, smem, s>>>(a, src, dst);
  }
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

template <int N, typename Real>
static mfx_status run_brick(const mfx_op* op, const Real* src, Real* dst, cudaStream_t s, const int32_t* skip) {
  constexpr int CB = BrickCB<N>::value;
  using Sh = BrickShape<N, CB>;
  static int blocks_per_sm = -1;
  const size_t smem = Sh::TABLE_BYTES + 3 * (size_t)Sh::CUBES * sizeof(Real);
  auto kern = brick_vmult_kernel<N, Real, CB>;
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
  MFX_CUDA_TRY(cudaMemsetAsync(dst, 0, sizeof(Real) * op->n_dofs, s));
  const int grid = (int)std::min<int64_t>(a.n_batches, (int64_t)device_sm_count() * blocks_per_sm);
  kern<<<grid, Sh::THREADS, smem, s>>>(a, src, dst);
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

template <int N>
int brick_cells_per_batch() { return BrickCB<N>::value; }

template <int N>
mfx_status launch_vmult_n(const mfx_op* op, mfx_prec prec, const void* src, void* dst, cudaStream_t s,
                          const int32_t* skip) {
  if (prec == MFX_F64) {
    if (op->structured) return run_brick<N, double>(op, (const double*)src, (double*)dst, s, skip);
    return run_vmult<N, double, false>(op, (const double*)src, (double*)dst, s, skip);
  }
  if (op->structured) return run_brick<N, float>(op, (const float*)src, (float*)dst, s, skip);
  return run_vmult<N, float, false>(op, (const float*)src, (float*)dst, s, skip);
}

}  // namespace mfx
